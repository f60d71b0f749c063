// Update batches on the device (Section 3.2: additions, deletions and
// modifications of vertices and edges in an evolving graph).
//
// A batch is a list of operations with sequential semantics. It is applied in
// parallel and exactly:
//   * vertex operations are grouped by vertex (stable radix sort), which gives
//     every vertex its final state and lets each EDGE_ADD check that both
//     endpoints are live at its own position in the batch;
//   * edge operations are grouped by edge key (u, w, l); for one key the
//     multiplicity after the batch is a fold over its operations in order
//     (ADD +1, DEL -1 floored at 0), started after the last deletion of u or w
//     (which removes every edge of the vertex at that moment);
//   * the out-CSR is rewritten once: initial edges incident to a deleted vertex
//     and the first r occurrences of a key that lost r copies are dropped, and
//     the added copies are appended to their rows.
// A batch that names an out-of-range vertex, an unknown kind, or an EDGE_ADD
// with an endpoint that is dead at that point is rejected before anything
// changes.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "prof.cuh"
#include "rows.cuh"

namespace bisim {

namespace {

constexpr uint64_t kSaltEdgeKey = 0x452821e638d01377ull;
constexpr unsigned kErrBadOp = 8u;
constexpr unsigned kErrDeadEndpoint = 16u;

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
unsigned grid_for(int64_t n, int threads) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(cdiv(n, threads), 1 << 20)));
}

__device__ __forceinline__ uint64_t edge_key_hash(int32_t u, int32_t w, int32_t l) {
    const uint64_t uw = (static_cast<uint64_t>(static_cast<uint32_t>(u)) << 32) | static_cast<uint32_t>(w);
    return mix64(uw ^ mix64(static_cast<uint64_t>(static_cast<uint32_t>(l)) ^ kSaltEdgeKey));
}

// ----------------------------------------------------------------------------- checks and grouping

__global__ void k_ops_check(const bisim_op* __restrict__ ops, int64_t nops, int32_t n, DevState* st,
                            uint32_t* __restrict__ vkey, uint64_t* __restrict__ vval) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nops;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const bisim_op o = ops[i];
        bool ok = o.kind >= BISIM_OP_EDGE_ADD && o.kind <= BISIM_OP_VERTEX_DEL && o.src >= 0 && o.src < n;
        const bool edge = o.kind == BISIM_OP_EDGE_ADD || o.kind == BISIM_OP_EDGE_DEL;
        if (edge) ok = ok && o.dst >= 0 && o.dst < n;
        if (!ok) atomicOr(&st->error, kErrBadOp);
        // vertex operations sort by vertex; edge operations go last, in batch order
        vkey[i] = (ok && !edge) ? static_cast<uint32_t>(o.src) : 0xffffffffu;
        vval[i] = static_cast<uint64_t>(i);
        if (ok && !edge) atomicAdd(&st->aux, 1ull);
        if (ok && o.kind == BISIM_OP_VERTEX_ADD) atomicAdd(&st->pairs, 1u);
    }
}

struct VertexOps {
    const uint32_t* key;     // sorted vertex of each vertex operation, [0, nv)
    const uint64_t* pos;     // its position in the batch (ascending within a vertex)
    int64_t nv;
    const bisim_op* ops;
    const uint8_t* alive0;   // state before the batch (null: all live)
};

__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t* a, int64_t n, uint32_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Is vertex x live just before position p of the batch?
__device__ bool alive_before(const VertexOps& V, int32_t x, uint64_t p) {
    const int64_t lo = lower_bound_u32(V.key, V.nv, static_cast<uint32_t>(x));
    int64_t hi = lo;
    while (hi < V.nv && V.key[hi] == static_cast<uint32_t>(x) && V.pos[hi] < p) ++hi;
    if (hi == lo) return V.alive0 == nullptr || V.alive0[x] != 0;
    return V.ops[V.pos[hi - 1]].kind == BISIM_OP_VERTEX_ADD;
}

// Position of the last deletion of x in the batch, or -1.
__device__ int64_t last_kill(const VertexOps& V, int32_t x) {
    const int64_t lo = lower_bound_u32(V.key, V.nv, static_cast<uint32_t>(x));
    int64_t last = -1;
    for (int64_t i = lo; i < V.nv && V.key[i] == static_cast<uint32_t>(x); ++i)
        if (V.ops[V.pos[i]].kind == BISIM_OP_VERTEX_DEL) last = static_cast<int64_t>(V.pos[i]);
    return last;
}

// Final state of every vertex named by a vertex operation.
// revived (nullable): live after the batch but dead before it or deleted in it.
__global__ void k_vertex_final(VertexOps V, uint8_t* __restrict__ alive, int32_t* __restrict__ vlabel,
                               uint8_t* __restrict__ killed, uint8_t* __restrict__ vchanged,
                               uint8_t* __restrict__ revived) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < V.nv;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint32_t x = V.key[i];
        if (V.ops[V.pos[i]].kind == BISIM_OP_VERTEX_DEL) killed[x] = 1;
        if (i + 1 < V.nv && V.key[i + 1] == x) continue;   // the last operation on x decides
        const bisim_op o = V.ops[V.pos[i]];
        const uint8_t was = alive[x];
        const int32_t lab = vlabel[x];
        if (o.kind == BISIM_OP_VERTEX_ADD) {
            alive[x] = 1;
            vlabel[x] = o.label;
            if (!was || lab != o.label) vchanged[x] = 1;
            if (revived && (!was || last_kill(V, static_cast<int32_t>(x)) >= 0)) revived[x] = 1;
        } else {
            alive[x] = 0;
            if (was) vchanged[x] = 1;
        }
    }
}

// Every EDGE_ADD needs both endpoints live at its position; also emits the
// edge-key hash of every edge operation for grouping. The vertex operations
// come first in the sorted order; their number is read on the device
// (st->aux), so this runs before the host has seen the batch's checks: an
// operation that fails them is skipped here and rejects the batch anyway.
__global__ void k_edge_ops(VertexOps V, const uint64_t* __restrict__ vpos, int64_t nops, int32_t n,
                           uint32_t* __restrict__ klo, uint32_t* __restrict__ khi, uint64_t* __restrict__ kval,
                           DevState* st) {
    V.nv = static_cast<int64_t>(*reinterpret_cast<const volatile unsigned long long*>(&st->aux));
    const int64_t ne = nops - V.nv;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < ne;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint64_t p = vpos[V.nv + j];
        const bisim_op o = V.ops[p];
        const bool valid = (o.kind == BISIM_OP_EDGE_ADD || o.kind == BISIM_OP_EDGE_DEL) && o.src >= 0 && o.src < n &&
                           o.dst >= 0 && o.dst < n;
        if (valid && o.kind == BISIM_OP_EDGE_ADD && (!alive_before(V, o.src, p) || !alive_before(V, o.dst, p)))
            atomicOr(&st->error, kErrDeadEndpoint);
        const uint64_t h = edge_key_hash(o.src, o.dst, o.label);
        klo[j] = static_cast<uint32_t>(h);
        khi[j] = static_cast<uint32_t>(h >> 32);
        kval[j] = p;
    }
}

// Key-hash halves of edge operations given in some order of positions.
__global__ void k_key_halves(const bisim_op* __restrict__ ops, const uint64_t* __restrict__ pos, int64_t ne,
                             uint32_t* __restrict__ lo, uint32_t* __restrict__ hi) {
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < ne;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const bisim_op o = ops[pos[j]];
        const uint64_t h = edge_key_hash(o.src, o.dst, o.label);
        if (lo) lo[j] = static_cast<uint32_t>(h);
        if (hi) hi[j] = static_cast<uint32_t>(h >> 32);
    }
}

struct AddRec {
    int32_t u, w, l, pad;
};

// A small open-addressing table of the batch's distinct edge keys (u, w, l):
// per key the copies present before the batch (c0), the copies to remove and
// the copies already marked for removal.
struct KeyTable {
    int32_t* u;
    int32_t* w;
    int32_t* l;
    int32_t* used;
    int32_t* c0;
    int32_t* rem;
    int32_t* taken;
    int32_t* hdel;     // the key has an EDGE_DEL in the batch (only then do its old copies matter)
    uint32_t mask;
};

__device__ __forceinline__ uint32_t key_home(int32_t u, int32_t w, int32_t l, uint32_t mask) {
    return static_cast<uint32_t>(edge_key_hash(u, w, l)) & mask;
}

__device__ int64_t key_insert(const KeyTable& T, int32_t u, int32_t w, int32_t l) {
    uint32_t pos = key_home(u, w, l, T.mask);
    for (uint32_t probe = 0; probe <= T.mask; ++probe) {
        if (atomicCAS(&T.used[pos], 0, 1) == 0) {
            T.u[pos] = u;
            T.w[pos] = w;
            T.l[pos] = l;
            return pos;
        }
        pos = (pos + 1) & T.mask;
    }
    return -1;
}

__device__ __forceinline__ int64_t key_find(const KeyTable& T, int32_t u, int32_t w, int32_t l) {
    uint32_t pos = key_home(u, w, l, T.mask);
    for (uint32_t probe = 0; probe <= T.mask; ++probe) {
        if (!T.used[pos]) return -1;
        if (T.u[pos] == u && T.w[pos] == w && T.l[pos] == l) return pos;
        pos = (pos + 1) & T.mask;
    }
    return -1;
}

// Every distinct key of the batch's edge operations enters the table once.
__global__ void k_keys_insert(const bisim_op* __restrict__ ops, const uint32_t* __restrict__ khi,
                              const uint32_t* __restrict__ klo, const uint64_t* __restrict__ kpos, int64_t ne,
                              KeyTable T, int64_t* __restrict__ keyslot, unsigned* err) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < ne;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const bisim_op o = ops[kpos[i]];
        // first appearance of this full key within its run of equal hashes
        bool first = true;
        for (int64_t b = i - 1; b >= 0 && khi[b] == khi[i] && klo[b] == klo[i]; --b) {
            const bisim_op ob = ops[kpos[b]];
            if (ob.src == o.src && ob.dst == o.dst && ob.label == o.label) { first = false; break; }
        }
        if (!first) { keyslot[i] = -1; continue; }
        const int64_t slot = key_insert(T, o.src, o.dst, o.label);
        if (slot < 0) atomicOr(err, 32u);
        keyslot[i] = slot;
    }
}

// Copies of every batch key present before the batch (one pass over the edges).
__global__ void k_keys_count(const int32_t* __restrict__ esrc, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ elab, int64_t m, KeyTable T) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t k = key_find(T, esrc[e], col[e], elab[e]);
        if (k >= 0) atomicAdd(&T.c0[k], 1);
    }
}

// One thread per distinct key: fold its operations in batch order, starting
// after the last deletion of an endpoint, and record the net change.
__global__ void k_fold_keys(VertexOps V, const uint32_t* __restrict__ khi, const uint32_t* __restrict__ klo,
                            const uint64_t* __restrict__ kpos, int64_t ne, const int64_t* __restrict__ keyslot,
                            KeyTable T, const uint8_t* __restrict__ killed, AddRec* __restrict__ add,
                            unsigned long long* __restrict__ counters, uint8_t* __restrict__ rowchg) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < ne;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t slot = keyslot[i];
        if (slot < 0) continue;                                // not the first appearance of its key
        const bisim_op oa = V.ops[kpos[i]];
        const int32_t u = oa.src, w = oa.dst, l = oa.label;
        const bool dropped = killed[u] || killed[w];           // initial copies go with the deletion
        int64_t end = i;
        while (end < ne && khi[end] == khi[i] && klo[end] == klo[i]) ++end;
        // a key that is only deleted removes one copy per deletion, as far as copies
        // exist: an old count at least its number of operations gives exactly that
        // (the row-store path does not count such keys; the removal stops when the
        // row has no copy left)
        const int c0 = dropped ? 0 : (T.hdel[slot] == 1 ? static_cast<int>(end - i) : T.c0[slot]);
        const int64_t lk = max(last_kill(V, u), last_kill(V, w));
        int c = c0;
        for (int64_t b = i; b < end; ++b) {
            const uint64_t p = kpos[b];
            const bisim_op ob = V.ops[p];
            if (ob.src != u || ob.dst != w || ob.label != l) continue;
            if (static_cast<int64_t>(p) < lk) continue;         // before the last deletion: no effect
            if (ob.kind == BISIM_OP_EDGE_ADD) ++c;
            else if (c > 0) --c;
        }
        const int adds = dropped ? c : max(c - c0, 0);
        const int removes = dropped ? 0 : max(c0 - c, 0);
        T.rem[slot] = removes;
        if (adds > 0) {
            const unsigned long long base = atomicAdd(&counters[1], static_cast<unsigned long long>(adds));
            for (int q = 0; q < adds; ++q) add[base + q] = AddRec{u, w, l, 0};
        }
        if (adds > 0 || removes > 0) rowchg[u] = 1;
    }
}

// ----------------------------------------------------------------------------- CSR rewrite

// Which edges survive the batch: not incident to a deleted vertex, and not one
// of the copies a key loses (any copies of one key are interchangeable).
__global__ void k_count_kept(const int32_t* __restrict__ esrc, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ elab, int64_t m, const uint8_t* __restrict__ killed,
                             KeyTable T, int use_table, uint8_t* __restrict__ keepf, int32_t* __restrict__ kept,
                             uint8_t* __restrict__ rowdirty, uint8_t* __restrict__ rowchg) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; e0 < m; e0 += stride) {
        const int64_t e = e0 + threadIdx.x;
        int32_t u = -1;
        bool keep = false;
        if (e < m) {
            u = esrc[e];
            const int32_t w = col[e];
            keep = !(killed[u] || killed[w]);
            if (keep && use_table) {
                const int64_t k = key_find(T, u, w, elab[e]);
                if (k >= 0 && T.rem[k] > 0 && atomicAdd(&T.taken[k], 1) < T.rem[k]) keep = false;
            }
            keepf[e] = keep ? 1 : 0;
            if (!keep) {
                rowdirty[u] = 1;
                rowchg[u] = 1;
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, u);
        const unsigned keepers = __ballot_sync(0xffffffffu, keep) & peers;
        if (e < m && (threadIdx.x & 31) == static_cast<unsigned>(__ffs(peers) - 1) && keepers)
            atomicAdd(&kept[u], __popc(keepers));
    }
}

__global__ void k_count_adds(const AddRec* __restrict__ add, int64_t nadd, int32_t* __restrict__ addcnt) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nadd;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        atomicAdd(&addcnt[add[i].u], 1);
}

__global__ void k_new_degree(const int32_t* __restrict__ kept, const int32_t* __restrict__ addcnt, int32_t n,
                             int64_t* __restrict__ deg) {
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < n) deg[v] = static_cast<int64_t>(kept[v]) + addcnt[v];
    if (v == n) deg[v] = 0;
}

// Kept edges move to the new CSR: rows without a dropped edge keep their order
// (offset shift); rows with drops take places from a per-row cursor, a warp
// reserving its share with one atomic (row order inside a row is irrelevant).
__global__ void k_copy_kept(const int32_t* __restrict__ esrc, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ elab, int64_t m, const int64_t* __restrict__ rp,
                            const int64_t* __restrict__ nrp, const uint8_t* __restrict__ rowdirty,
                            const uint8_t* __restrict__ keepf, int32_t* __restrict__ dcursor,
                            int32_t* __restrict__ ncol, int32_t* __restrict__ nelab, int32_t* __restrict__ nsrc) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; e0 < m; e0 += stride) {
        const int64_t e = e0 + threadIdx.x;
        int32_t u = -1;
        bool keep = false, dirty = false;
        if (e < m) {
            u = esrc[e];
            keep = keepf[e] != 0;
            dirty = rowdirty[u] != 0;
        }
        const bool via_cursor = keep && dirty;
        const int lane = static_cast<int>(threadIdx.x & 31);
        const unsigned peers = __match_any_sync(0xffffffffu, via_cursor ? u : -1);
        const unsigned takers = __ballot_sync(0xffffffffu, via_cursor) & peers;
        const int leader = via_cursor ? __ffs(takers) - 1 : lane;
        int base = 0;
        if (via_cursor && lane == leader) base = atomicAdd(&dcursor[u], __popc(takers));
        base = __shfl_sync(0xffffffffu, base, leader);
        int64_t p = -1;
        if (via_cursor) {
            p = nrp[u] + base + __popc(takers & ((1u << lane) - 1u));
        } else if (keep) {
            p = nrp[u] + (e - rp[u]);
        }
        if (p >= 0) {
            ncol[p] = col[e];
            nelab[p] = elab[e];
            nsrc[p] = u;
        }
    }
}

// Appended copies: one thread per record; records of a row are counted in order.
__global__ void k_place_adds(const AddRec* __restrict__ add, int64_t nadd, const int64_t* __restrict__ nrp,
                             const int32_t* __restrict__ kept, int32_t* __restrict__ cursor,
                             int32_t* __restrict__ ncol, int32_t* __restrict__ nelab, int32_t* __restrict__ nsrc) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nadd;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const AddRec a = add[i];
        const int slot = atomicAdd(&cursor[a.u], 1);
        const int64_t p = nrp[a.u] + kept[a.u] + slot;
        ncol[p] = a.w;
        nelab[p] = a.l;
        nsrc[p] = a.u;
    }
}

__global__ void k_fill_src(const int64_t* __restrict__ rp, int32_t n, int32_t* __restrict__ esrc) {
    // one warp per vertex
    const int64_t v = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (v >= n) return;
    for (int64_t e = rp[v] + (threadIdx.x & 31); e < rp[v + 1]; e += 32) esrc[e] = static_cast<int32_t>(v);
}

// ----------------------------------------------------------------------------- row-store edits

// Operation kinds per key: bit 0 a deletion, bit 1 an addition. A key that is
// only added to ends with its old copies plus its adds whatever the old count;
// one that is only deleted removes a copy per deletion while copies last; only
// keys with both need their old copies counted.
__global__ void k_mark_kinds(const bisim_op* __restrict__ ops, const uint64_t* __restrict__ kpos, int64_t ne,
                             KeyTable T) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < ne;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const bisim_op o = ops[kpos[i]];
        const int64_t k = key_find(T, o.src, o.dst, o.label);
        if (k >= 0) atomicOr(&T.hdel[k], o.kind == BISIM_OP_EDGE_DEL ? 1 : 2);
    }
}

// Source rows of the keys with a deletion (rows_del) and of the keys with both
// kinds (rows_mix), each listed once per list (xmark is kept zero between batches).
// Their targets are also flagged in the bitmap `dmark` (kept zero between
// batches), which lets the row scans skip most entries without a table lookup.
__global__ void k_key_rows(const int64_t* __restrict__ keyslot, int64_t ne, KeyTable T, uint32_t* __restrict__ xmark,
                           uint32_t* __restrict__ dmark, int32_t* __restrict__ rows_del,
                           int32_t* __restrict__ rows_mix, unsigned* __restrict__ n_rows) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < ne;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (keyslot[i] < 0) continue;
        const int kinds = T.hdel[keyslot[i]];
        if (!(kinds & 1)) continue;
        const int32_t u = T.u[keyslot[i]];
        const int32_t w = T.w[keyslot[i]];
        atomicOr(&dmark[w >> 5], 1u << (w & 31));
        const unsigned old = atomicOr(&xmark[u], kinds == 3 ? 3u : 1u);
        if (!(old & 1u)) rows_del[atomicAdd(&n_rows[0], 1u)] = u;
        if (kinds == 3 && !(old & 2u)) rows_mix[atomicAdd(&n_rows[1], 1u)] = u;
    }
}

__global__ void k_clear_dmark(const int64_t* __restrict__ keyslot, int64_t ne, KeyTable T,
                              uint32_t* __restrict__ dmark) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < ne;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        if (keyslot[i] >= 0 && (T.hdel[keyslot[i]] & 1)) dmark[T.w[keyslot[i]] >> 5] = 0u;
}

__global__ void k_rows_to_tasks(const int32_t* __restrict__ rows, const unsigned* __restrict__ n_rows, StoreView S,
                                uint32_t* __restrict__ xmark, int clear, TierLists L) {
    const unsigned count = *reinterpret_cast<const volatile unsigned*>(n_rows);
    for (unsigned b0 = blockIdx.x * blockDim.x; b0 < count; b0 += gridDim.x * blockDim.x) {
        const unsigned i = b0 + threadIdx.x;
        bool has = false;
        RowTask t{0, 0, 0};
        if (i < count) {
            const int32_t u = rows[i];
            has = true;
            t = RowTask{S.xro[u], S.xlen[u], u};
            if (clear) xmark[u] = 0u;
        }
        tier_push(L, has, t);
    }
}

// Copies of each batch key present before the batch: every touched source row
// is scanned once and its entries looked up in the batch's key table. An
// entry into a vertex that was dead before the batch is not an edge.
__device__ __forceinline__ bool dmarked(const uint32_t* dmark, int32_t w) {
    return (dmark[w >> 5] >> (w & 31)) & 1u;
}

struct KeyCountRows {
    const unsigned long long* xpe;
    const uint8_t* alive0;
    const uint32_t* dmark;
    KeyTable T;
    __device__ void operator()(const RowTask& t, int64_t e, bool in) const {
        if (!in) return;
        const unsigned long long x = xpe[e];
        if (x == kRowTomb) return;
        const int32_t w = static_cast<int32_t>(static_cast<uint32_t>(x));
        if (!dmarked(dmark, w) || !alive0[w]) return;
        const int64_t k = key_find(T, t.arg, w, static_cast<int32_t>(x >> 32));
        if (k >= 0 && T.hdel[k] == 3) atomicAdd(&T.c0[k], 1);
    }
};

// Deletes the copies the fold removed (any copies of a key are interchangeable).
struct KeyRemoveRows {
    unsigned long long* xpe;
    const uint32_t* dmark;
    KeyTable T;
    __device__ void operator()(const RowTask& t, int64_t e, bool in) const {
        if (!in) return;
        const unsigned long long x = xpe[e];
        if (x == kRowTomb) return;
        const int32_t w = static_cast<int32_t>(static_cast<uint32_t>(x));
        if (!dmarked(dmark, w)) return;
        const int64_t k = key_find(T, t.arg, w, static_cast<int32_t>(x >> 32));
        if (k >= 0 && T.rem[k] > 0 && atomicAdd(&T.taken[k], 1) < T.rem[k]) xpe[e] = kRowTomb;
    }
};

// KeyRemoveRows for the grid tier (rows longer than kCtaTierMax, the hubs).
// The rows are cut into chunks of kLongChunk entries dealt round-robin to the
// CTAs across all rows (so every CTA stays busy whatever the row lengths), and
// every thread loads its kLongRun consecutive entries before it looks at any.
constexpr int kLongRun = 8;
constexpr int64_t kLongChunk = static_cast<int64_t>(kTierThreads) * kLongRun;
__global__ void __launch_bounds__(kTierThreads) k_remove_long(const TierLists L, unsigned long long* __restrict__ xpe,
                                                              const uint32_t* __restrict__ dmark, KeyTable T) {
    const unsigned c2 = *reinterpret_cast<volatile unsigned*>(&L.cnt[2]);
    const int64_t G = gridDim.x;
    int64_t first = 0;                               // global index of the row's first chunk
    for (unsigned i = 0; i < c2; ++i) {
        const RowTask t = L.t[2][i];
        const int64_t nch = (t.len + kLongChunk - 1) / kLongChunk;
        int64_t k = (static_cast<int64_t>(blockIdx.x) - first) % G;
        if (k < 0) k += G;
        for (; k < nch; k += G) {
            const int64_t j0 = k * kLongChunk + static_cast<int64_t>(threadIdx.x) * kLongRun;
            unsigned long long x[kLongRun];
#pragma unroll
            for (int q = 0; q < kLongRun; ++q) x[q] = j0 + q < t.len ? xpe[t.off + j0 + q] : kRowTomb;
#pragma unroll
            for (int q = 0; q < kLongRun; ++q) {
                if (x[q] == kRowTomb) continue;
                const int32_t w = static_cast<int32_t>(static_cast<uint32_t>(x[q]));
                if (!dmarked(dmark, w)) continue;
                const int64_t key = key_find(T, t.arg, w, static_cast<int32_t>(x[q] >> 32));
                if (key >= 0 && T.rem[key] > 0 && atomicAdd(&T.taken[key], 1) < T.rem[key])
                    xpe[t.off + j0 + q] = kRowTomb;
            }
        }
        first += nch;
    }
}

// In-row tasks of every vertex deleted or brought back by the batch (the last
// operation of each named vertex files it). With `need` set, only adds the
// in-row lengths of the revived vertices there.
__global__ void k_vertex_tasks(VertexOps V, const uint8_t* __restrict__ killed, const uint8_t* __restrict__ revived,
                               StoreView S, TierLists L, unsigned long long* need) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t b0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; b0 < V.nv; b0 += stride) {
        const int64_t i = b0 + threadIdx.x;
        bool has = false;
        RowTask t{0, 0, 0};
        if (i < V.nv && (i + 1 == V.nv || V.key[i + 1] != V.key[i])) {
            const int32_t x = static_cast<int32_t>(V.key[i]);
            if (need) {
                if (revived[x]) atomicAdd(need, static_cast<unsigned long long>(S.ylen[x]));
            } else if (killed[x] || revived[x]) {
                has = true;
                t = RowTask{S.yro[x], S.ylen[x], x};
            }
        }
        if (!need) tier_push(L, has, t);
    }
}

// Sources of a deleted vertex lose an out-edge; the out-rows of a revived
// vertex's former sources are searched for entries left pointing at it.
struct VertexSources {
    const int32_t* ype;
    const uint8_t* killed;
    const uint8_t* revived;
    uint8_t* rowchg;
    StoreView S;
    TierLists P;
    __device__ void operator()(const RowTask& t, int64_t e, bool in) const {
        const int32_t x = t.arg;
        int32_t u = 0;
        if (in) {
            u = ype[e];
            if (killed[x]) rowchg[u] = 1;
        }
        const bool purge = in && revived[x] != 0;
        RowTask pt{0, 0, x};
        if (purge) pt = RowTask{S.xro[u], S.xlen[u], x};
        tier_push(P, purge, pt);
    }
};

struct PurgeTarget {
    unsigned long long* xpe;
    __device__ void operator()(const RowTask& t, int64_t e, bool in) const {
        if (in && static_cast<uint32_t>(xpe[e]) == static_cast<uint32_t>(t.arg)) xpe[e] = kRowTomb;
    }
};

// A deleted vertex's out-row empties, and its out-edges count as changed: a
// vertex deleted and added again in one batch with its old label is live
// before and after and keeps its label, so only this flag puts it into the
// frontiers above level 0. A revived vertex's in-row starts afresh (its former
// sources were purged).
__global__ void k_vertex_rows(VertexOps V, const uint8_t* __restrict__ killed, const uint8_t* __restrict__ revived,
                              StoreView S, uint8_t* __restrict__ rowchg) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < V.nv;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (i + 1 < V.nv && V.key[i + 1] == V.key[i]) continue;
        const int32_t x = static_cast<int32_t>(V.key[i]);
        if (killed[x]) {
            S.xlen[x] = 0;
            rowchg[x] = 1;
        }
        if (revived[x]) S.ylen[x] = 0;
    }
}

// Adds per out-row and per in-row; every row that receives one is listed once.
__global__ void k_add_rows(const AddRec* __restrict__ add, const unsigned long long* __restrict__ nadd,
                           int32_t* __restrict__ addo, int32_t* __restrict__ addi, int32_t* __restrict__ touched_o,
                           int32_t* __restrict__ touched_i, unsigned* __restrict__ n_touched) {
    const int64_t count = static_cast<int64_t>(*reinterpret_cast<const volatile unsigned long long*>(nadd));
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const AddRec a = add[i];
        if (atomicAdd(&addo[a.u], 1) == 0) touched_o[atomicAdd(&n_touched[0], 1u)] = a.u;
        if (atomicAdd(&addi[a.w], 1) == 0) touched_i[atomicAdd(&n_touched[1], 1u)] = a.w;
    }
}

struct RowMove {
    int64_t off;     // new offset (-1: the row stays)
    int32_t cap;
    int32_t len;     // entries copied so far
};

// A row that cannot take its adds moves to the pool's tail with room for half
// as much again. A move that would pass the pool's end is not made (the tail
// still advances, so the host sees the overflow and rebuilds the store before
// any add is placed); `wanted` sums the room all moves asked for.
__global__ void k_plan_rows(const int32_t* __restrict__ touched, const unsigned* __restrict__ n_touched,
                            const int32_t* __restrict__ addc, const int32_t* __restrict__ len,
                            const int32_t* __restrict__ cap, int64_t* __restrict__ tail, int64_t pool,
                            int64_t* __restrict__ wanted, RowMove* __restrict__ moves) {
    const unsigned count = *reinterpret_cast<const volatile unsigned*>(n_touched);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const int32_t v = touched[i];
        const int64_t need = static_cast<int64_t>(len[v]) + addc[v];
        RowMove mv{-1, 0, 0};
        if (need > cap[v]) {
            const int64_t want = need + need / 2 + 8;
            const int64_t nc = want < 0x7fffffff ? want : 0x7fffffff;
            const int64_t off = static_cast<int64_t>(atomicAdd(reinterpret_cast<unsigned long long*>(tail),
                                                               static_cast<unsigned long long>(nc)));
            atomicAdd(reinterpret_cast<unsigned long long*>(wanted), static_cast<unsigned long long>(nc));
            if (off + nc <= pool) mv = RowMove{off, static_cast<int32_t>(nc), 0};
        }
        moves[i] = mv;
    }
}

__global__ void k_move_tasks(const int32_t* __restrict__ touched, const unsigned* __restrict__ n_touched,
                             const RowMove* __restrict__ moves, const int64_t* __restrict__ ro,
                             const int32_t* __restrict__ len, TierLists L) {
    const unsigned count = *reinterpret_cast<const volatile unsigned*>(n_touched);
    for (unsigned b0 = blockIdx.x * blockDim.x; b0 < count; b0 += gridDim.x * blockDim.x) {
        const unsigned i = b0 + threadIdx.x;
        bool has = false;
        RowTask t{0, 0, static_cast<int32_t>(i)};
        if (i < count && moves[i].off >= 0) {
            has = true;
            t.off = ro[touched[i]];
            t.len = len[touched[i]];
        }
        tier_push(L, has, t);
    }
}

// Copies the live entries of a moving out-row (deleted entries and edges into
// dead vertices are dropped).
struct MoveOut {
    unsigned long long* xpe;
    const uint8_t* alive;
    RowMove* moves;
    __device__ void operator()(const RowTask& t, int64_t e, bool in) const {
        unsigned long long x = 0;
        bool ok = false;
        if (in) {
            x = xpe[e];
            ok = x != kRowTomb && alive[static_cast<int32_t>(static_cast<uint32_t>(x))];
        }
        const unsigned b = __ballot_sync(0xffffffffu, ok);
        if (b == 0u) return;
        int base = 0;
        if ((threadIdx.x & 31u) == 0u) base = atomicAdd(&moves[t.arg].len, __popc(b));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (ok) xpe[moves[t.arg].off + base + __popc(b & ((1u << (threadIdx.x & 31u)) - 1u))] = x;
    }
};

// The same for a moving in-row (entries of dead sources are dropped).
struct MoveIn {
    int32_t* ype;
    const uint8_t* alive;
    RowMove* moves;
    __device__ void operator()(const RowTask& t, int64_t e, bool in) const {
        int32_t x = 0;
        bool ok = false;
        if (in) {
            x = ype[e];
            ok = alive[x] != 0;
        }
        const unsigned b = __ballot_sync(0xffffffffu, ok);
        if (b == 0u) return;
        int base = 0;
        if ((threadIdx.x & 31u) == 0u) base = atomicAdd(&moves[t.arg].len, __popc(b));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (ok) ype[moves[t.arg].off + base + __popc(b & ((1u << (threadIdx.x & 31u)) - 1u))] = x;
    }
};

__global__ void k_finish_moves(const int32_t* __restrict__ touched, const unsigned* __restrict__ n_touched,
                               const RowMove* __restrict__ moves, int64_t* __restrict__ ro, int32_t* __restrict__ len,
                               int32_t* __restrict__ cap) {
    const unsigned count = *reinterpret_cast<const volatile unsigned*>(n_touched);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const RowMove mv = moves[i];
        if (mv.off < 0) continue;
        const int32_t v = touched[i];
        ro[v] = mv.off;
        len[v] = mv.len;
        cap[v] = mv.cap;
    }
}

// Appends every added copy to its out-row and its target's in-row.
__global__ void k_place_adds_rows(const AddRec* __restrict__ add, const unsigned long long* __restrict__ nadd,
                                  StoreView S) {
    const int64_t count = static_cast<int64_t>(*reinterpret_cast<const volatile unsigned long long*>(nadd));
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const AddRec a = add[i];
        const int32_t p = atomicAdd(&S.xlen[a.u], 1);
        S.xpe[S.xro[a.u] + p] = pack_edge(a.l, a.w);
        const int32_t q = atomicAdd(&S.ylen[a.w], 1);
        S.ype[S.yro[a.w] + q] = a.u;
    }
}

__global__ void k_clear_rows(const int32_t* __restrict__ touched, const unsigned* __restrict__ n_touched,
                             int32_t* __restrict__ addc) {
    const unsigned count = *reinterpret_cast<const volatile unsigned*>(n_touched);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        addc[touched[i]] = 0;
}

}  // namespace

// Frees one buffer owned by ctx (stream-ordered).
void ctx_free(bisim_ctx* ctx, void* p, size_t bytes, cudaStream_t s) {
    if (p == nullptr) return;
    auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), p);
    if (it != ctx->allocs.end()) ctx->allocs.erase(it);
    ctx->device_bytes -= static_cast<int64_t>(bytes);
    cudaFreeAsync(p, s);
}

// Per-edge source array for the current CSR (needed to rewrite it edge-parallel).
bisim_status ensure_edge_sources(bisim_ctx* ctx, cudaStream_t s) {
    if (ctx->esrc != nullptr) return BISIM_OK;
    bisim_status st = ensure_vertex_csr(ctx, s);
    if (st != BISIM_OK) return st;
    cudaError_t e;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->esrc), sizeof(int32_t) * std::max<int64_t>(ctx->m, 1), s)))
        return cuda_error(ctx, e, "alloc edge sources");
    ctx->esrc_cap = std::max<int64_t>(ctx->m, 1);
    if (ctx->n > 0) {
        BISIM_SITE(site, "edge_sources");
        Launch L(site, s, ctx->n, ctx->m, 8.0 * ctx->n + 4.0 * ctx->m);
        k_fill_src<<<grid_for(static_cast<int64_t>(ctx->n) * 32, 256), 256, 0, s>>>(ctx->row_ptr, ctx->n, ctx->esrc);
    }
    if (!ctx->alive) {
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->alive), std::max(ctx->n, 1), s)))
            return cuda_error(ctx, e, "alloc alive");
        cudaMemsetAsync(ctx->alive, 1, std::max(ctx->n, 1), s);
    }
    return BISIM_OK;
}

namespace {

// Scratch and results of the steps both batch paths share.
struct Batch {
    char* base = nullptr;
    VertexOps V{};
    int64_t nv = 0, ne = 0, vadds = 0;
    const uint32_t* skhi = nullptr;
    const uint32_t* sklo = nullptr;
    const uint64_t* skp = nullptr;
    KeyTable T{};
    int64_t* keyslot = nullptr;
    AddRec* add = nullptr;
    unsigned long long* counters = nullptr;
    int64_t* tmp = nullptr;
    char* extra = nullptr;           // the path's own scratch
};

// The steps both paths share: checks (nothing of the graph changes before they
// pass), grouping by vertex and by edge key, the final state of every named
// vertex, and the batch's key table. `extra` bytes of path-specific scratch
// follow the shared buffers; `alive0` (nullable) receives the liveness before
// the batch and `revived` (nullable) the vertices that come back.
bisim_status batch_begin(bisim_ctx* ctx, const bisim_op* d_ops, int64_t nops, size_t extra, uint8_t* vchanged,
                         uint8_t* killed, uint8_t* revived, uint8_t* alive0, Batch& B, cudaStream_t s) {
    const int32_t n = ctx->n;
    cudaError_t e;
    const size_t tmpw = std::max(radix_temp_words(std::max<int64_t>(nops, 1)), scan_temp_words(n + 1));
    const size_t nb = static_cast<size_t>(std::max<int64_t>(nops, 1));
    uint32_t tsize = 64;
    while (tsize < 2u * static_cast<uint32_t>(std::min<int64_t>(nops, 1 << 30))) tsize <<= 1;
    size_t bytes = 0;
    auto need = [&](size_t b) { bytes += (b + 255) & ~size_t(255); };
    need(4 * nb); need(4 * nb); need(8 * nb); need(8 * nb);          // vertex-op keys / values (x2)
    need(4 * nb); need(4 * nb); need(4 * nb); need(4 * nb);          // edge key halves (x2 each)
    need(8 * nb); need(8 * nb); need(8 * nb); need(8 * nb);          // edge positions (x4)
    need(sizeof(AddRec) * nb); need(8 * nb);                          // additions, key slots
    for (int q = 0; q < 8; ++q) need(4 * static_cast<size_t>(tsize)); // key table
    need(8 * 4);
    need(8 * tmpw);
    need(extra);
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&B.base), bytes, s))) return cuda_error(ctx, e, "alloc update scratch");
    char* scratch = B.base;
    auto carve = [&](size_t b) { char* p = scratch; scratch += (b + 255) & ~size_t(255); return p; };
    uint32_t* vk0 = reinterpret_cast<uint32_t*>(carve(4 * nb));
    uint32_t* vk1 = reinterpret_cast<uint32_t*>(carve(4 * nb));
    uint64_t* vv0 = reinterpret_cast<uint64_t*>(carve(8 * nb));
    uint64_t* vv1 = reinterpret_cast<uint64_t*>(carve(8 * nb));
    uint32_t* klo0 = reinterpret_cast<uint32_t*>(carve(4 * nb));
    uint32_t* klo1 = reinterpret_cast<uint32_t*>(carve(4 * nb));
    uint32_t* khi0 = reinterpret_cast<uint32_t*>(carve(4 * nb));
    uint32_t* khi1 = reinterpret_cast<uint32_t*>(carve(4 * nb));
    uint64_t* kp0 = reinterpret_cast<uint64_t*>(carve(8 * nb));
    uint64_t* kp1 = reinterpret_cast<uint64_t*>(carve(8 * nb));
    uint64_t* kp2 = reinterpret_cast<uint64_t*>(carve(8 * nb));
    uint64_t* kp3 = reinterpret_cast<uint64_t*>(carve(8 * nb));
    B.add = reinterpret_cast<AddRec*>(carve(sizeof(AddRec) * nb));
    B.keyslot = reinterpret_cast<int64_t*>(carve(8 * nb));
    int32_t* tab_arrays[8];
    for (int q = 0; q < 8; ++q) tab_arrays[q] = reinterpret_cast<int32_t*>(carve(4 * static_cast<size_t>(tsize)));
    B.T = KeyTable{tab_arrays[0], tab_arrays[1], tab_arrays[2], tab_arrays[3], tab_arrays[4], tab_arrays[5],
                   tab_arrays[6], tab_arrays[7], tsize - 1};
    B.counters = reinterpret_cast<unsigned long long*>(carve(8 * 4));
    B.tmp = reinterpret_cast<int64_t*>(carve(8 * tmpw));
    B.extra = carve(extra);
    auto fail = [&](bisim_status code, const char* msg) {
        cudaFreeAsync(B.base, s);
        B.base = nullptr;
        return set_error(ctx, code, msg);
    };

    BISIM_SITE(site_ops, "update_ops");
    // 1. check kinds and ranges; group vertex operations by vertex
    cudaMemsetAsync(ctx->dstate, 0, sizeof(DevState), s);
    {
        Launch L(site_ops, s, 0, 0, 16.0 * nops);
        k_ops_check<<<grid_for(nops, 256), 256, 0, s>>>(d_ops, nops, n, ctx->dstate, vk0, vv0);
    }
    const int which = radix_sort_pairs(vk0, vv0, vk1, vv1, nops, 32, B.tmp, s, "update_radix");
    const uint32_t* vkey = which ? vk1 : vk0;
    const uint64_t* vpos = which ? vv1 : vv0;
    // 2. EDGE_ADD liveness and edge-key hashes (before the host looks: one read-back
    // covers both checks)
    if (nops > 0) {
        Launch L(site_ops, s, 0, 0, 24.0 * nops);
        B.V = VertexOps{vkey, vpos, 0, d_ops, ctx->alive};
        k_edge_ops<<<grid_for(nops, 256), 256, 0, s>>>(B.V, vpos, nops, n, klo0, khi0, kp0, ctx->dstate);
    }
    cudaMemcpyAsync(ctx->hstate, ctx->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) {
        cudaFreeAsync(B.base, s);
        B.base = nullptr;
        return cuda_error(ctx, e, "check update batch");
    }
    if (ctx->hstate->error & kErrBadOp) return fail(BISIM_EINVAL, "update batch names an out-of-range vertex or an unknown kind");
    if (ctx->hstate->error & kErrDeadEndpoint) return fail(BISIM_EINVAL, "EDGE_ADD with an endpoint that is dead at that point of the batch");
    B.nv = static_cast<int64_t>(ctx->hstate->aux);
    B.vadds = static_cast<int64_t>(ctx->hstate->pairs);
    B.ne = nops - B.nv;
    B.V = VertexOps{vkey, vpos, B.nv, d_ops, ctx->alive};
    const int64_t nv = B.nv, ne = B.ne;

    // ---- from here on the batch is valid and the graph changes ----
    // stable LSD sort of the edge operations by key hash: low half, then high
    // half; operations of one key stay in batch order
    B.skhi = khi0;
    B.sklo = klo0;
    B.skp = kp0;
    if (ne > 0) {
        const int wa = radix_sort_pairs(klo0, kp0, klo1, kp1, ne, 32, B.tmp, s, "update_radix");
        const uint64_t* posA = wa ? kp1 : kp0;
        k_key_halves<<<grid_for(ne, 256), 256, 0, s>>>(d_ops, posA, ne, nullptr, khi0);
        cudaMemcpyAsync(kp2, posA, 8 * ne, cudaMemcpyDeviceToDevice, s);
        const int wb = radix_sort_pairs(khi0, kp2, khi1, kp3, ne, 32, B.tmp, s, "update_radix");
        B.skhi = wb ? khi1 : khi0;
        B.skp = wb ? kp3 : kp2;
        k_key_halves<<<grid_for(ne, 256), 256, 0, s>>>(d_ops, B.skp, ne, klo0, nullptr);
        B.sklo = klo0;
    }
    cudaMemsetAsync(killed, 0, n + 1, s);
    cudaMemsetAsync(B.counters, 0, 8 * 4, s);
    for (int q = 3; q < 8; ++q) cudaMemsetAsync(tab_arrays[q], 0, 4 * static_cast<size_t>(tsize), s);
    if (alive0 && n > 0) cudaMemcpyAsync(alive0, ctx->alive, n, cudaMemcpyDeviceToDevice, s);
    if (nv > 0) {
        Launch L(site_ops, s, 0, 0, 16.0 * nv);
        k_vertex_final<<<grid_for(nv, 256), 256, 0, s>>>(B.V, ctx->alive, ctx->vlabel, killed, vchanged, revived);
    }
    if (ne > 0) {
        Launch L(site_ops, s, 0, 0, 32.0 * ne);
        k_keys_insert<<<grid_for(ne, 256), 256, 0, s>>>(d_ops, B.skhi, B.sklo, B.skp, ne, B.T, B.keyslot,
                                                       &ctx->dstate->error);
    }
    return BISIM_OK;
}

// Net effect of every key: copies to remove and copies to add (after the key
// table's c0 holds the copies present before the batch).
void fold_keys(const Batch& B, const uint8_t* killed, uint8_t* rowchg, cudaStream_t s) {
    if (B.ne <= 0) return;
    BISIM_SITE(site_ops, "update_ops");
    Launch L(site_ops, s, 0, 0, 32.0 * B.ne);
    k_fold_keys<<<grid_for(B.ne, 128), 128, 0, s>>>(B.V, B.skhi, B.sklo, B.skp, B.ne, B.keyslot, B.T, killed, B.add,
                                                   B.counters, rowchg);
}

}  // namespace

bisim_status apply_ops_to_graph(bisim_ctx* ctx, const bisim_op* d_ops, int64_t nops, uint8_t* vchanged,
                                uint8_t* rowchg, uint8_t* killed, cudaStream_t s) {
    const int32_t n = ctx->n;
    const int64_t m = ctx->m;
    cudaError_t e;
    bisim_status st;
    if ((st = ensure_edge_sources(ctx, s)) != BISIM_OK) return st;
    size_t extra = 0;
    auto need = [&](size_t b) { extra += (b + 255) & ~size_t(255); };
    need(std::max<int64_t>(m, 1));                                    // keep flags
    need(4 * (n + 1)); need(4 * (n + 1)); need(4 * (n + 1));          // kept, addcnt, cursor
    need(4 * (n + 1));                                                // dirty-row cursor
    need(1 * (n + 1));                                                // rowdirty
    need(8 * (n + 1));                                                // new degree
    Batch B;
    if ((st = batch_begin(ctx, d_ops, nops, extra, vchanged, killed, nullptr, nullptr, B, s)) != BISIM_OK) return st;
    char* scratch = B.extra;
    auto carve = [&](size_t b) { char* p = scratch; scratch += (b + 255) & ~size_t(255); return p; };
    uint8_t* keepf = reinterpret_cast<uint8_t*>(carve(std::max<int64_t>(m, 1)));
    int32_t* kept = reinterpret_cast<int32_t*>(carve(4 * (n + 1)));
    int32_t* addcnt = reinterpret_cast<int32_t*>(carve(4 * (n + 1)));
    int32_t* cursor = reinterpret_cast<int32_t*>(carve(4 * (n + 1)));
    int32_t* dcursor = reinterpret_cast<int32_t*>(carve(4 * (n + 1)));
    uint8_t* rowdirty = reinterpret_cast<uint8_t*>(carve(n + 1));
    int64_t* ndeg = reinterpret_cast<int64_t*>(carve(8 * (n + 1)));
    const int64_t ne = B.ne;
    KeyTable& T = B.T;
    BISIM_SITE(site_ops, "update_ops");
    if (ne > 0 && m > 0) {
        Launch L(site_ops, s, 0, m, 12.0 * m);
        k_keys_count<<<grid_for(m, 256), 256, 0, s>>>(ctx->esrc, ctx->col, ctx->elab, m, T);
    }
    fold_keys(B, killed, rowchg, s);
    unsigned long long hc[2] = {0, 0};
    cudaMemcpyAsync(hc, B.counters, sizeof(hc), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) { cudaFreeAsync(B.base, s); return cuda_error(ctx, e, "fold edge operations"); }
    const int64_t nadd = static_cast<int64_t>(hc[1]);
    AddRec* add = B.add;

    // 3. rewrite the CSR
    BISIM_SITE(site_csr, "update_csr");
    cudaMemsetAsync(kept, 0, 4 * (n + 1), s);
    cudaMemsetAsync(addcnt, 0, 4 * (n + 1), s);
    cudaMemsetAsync(cursor, 0, 4 * (n + 1), s);
    cudaMemsetAsync(dcursor, 0, 4 * (n + 1), s);
    cudaMemsetAsync(rowdirty, 0, n + 1, s);
    if (m > 0) {
        Launch L(site_csr, s, 0, m, 13.0 * m);
        k_count_kept<<<grid_for(m, 256), 256, 0, s>>>(ctx->esrc, ctx->col, ctx->elab, m, killed, T, ne > 0 ? 1 : 0,
                                                     keepf, kept, rowdirty, rowchg);
    }
    if (nadd > 0) {
        Launch L(site_csr, s, 0, 0, 16.0 * nadd);
        k_count_adds<<<grid_for(nadd, 256), 256, 0, s>>>(add, nadd, addcnt);
    }
    {
        Launch L(site_csr, s, n, 0, 16.0 * n);
        k_new_degree<<<grid_for(n + 1, 256), 256, 0, s>>>(kept, addcnt, n, ndeg);
    }
    int64_t* nrp = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&nrp), sizeof(int64_t) * (n + 1), s))) {
        cudaFreeAsync(B.base, s);
        return cuda_error(ctx, e, "alloc row_ptr");
    }
    exclusive_scan_i64(ndeg, nrp, n + 1, B.tmp, s);
    int64_t new_m = 0;
    cudaMemcpyAsync(&new_m, nrp + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) { cudaFreeAsync(B.base, s); cudaFreeAsync(nrp, s); return cuda_error(ctx, e, "size new CSR"); }
    int32_t *ncol = nullptr, *nelab = nullptr, *nsrc = nullptr;
    const size_t cap = static_cast<size_t>(std::max<int64_t>(new_m, 1));
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&ncol), 4 * cap, s)) ||
        (e = cudaMallocAsync(reinterpret_cast<void**>(&nelab), 4 * cap, s)) ||
        (e = cudaMallocAsync(reinterpret_cast<void**>(&nsrc), 4 * cap, s))) {
        cudaFreeAsync(B.base, s);
        return cuda_error(ctx, e, "alloc new CSR");
    }
    if (m > 0) {
        Launch L(site_csr, s, 0, m, 26.0 * m);
        k_copy_kept<<<grid_for(m, 256), 256, 0, s>>>(ctx->esrc, ctx->col, ctx->elab, m, ctx->row_ptr, nrp, rowdirty,
                                                    keepf, dcursor, ncol, nelab, nsrc);
    }
    if (nadd > 0) {
        Launch L(site_csr, s, 0, nadd, 24.0 * nadd);
        k_place_adds<<<grid_for(nadd, 256), 256, 0, s>>>(add, nadd, nrp, kept, cursor, ncol, nelab, nsrc);
    }
    // swap in the new CSR
    ctx_free(ctx, ctx->col, 4 * static_cast<size_t>(std::max<int64_t>(m, 1)), s);
    ctx_free(ctx, ctx->elab, 4 * static_cast<size_t>(std::max<int64_t>(m, 1)), s);
    ctx_free(ctx, ctx->esrc, 4 * static_cast<size_t>(ctx->esrc_cap), s);
    ctx->col = ncol;
    ctx->elab = nelab;
    ctx->esrc = nsrc;
    ctx->esrc_cap = static_cast<int64_t>(cap);
    for (void* p : {static_cast<void*>(ncol), static_cast<void*>(nelab), static_cast<void*>(nsrc)}) ctx->allocs.push_back(p);
    ctx->device_bytes += 12 * static_cast<int64_t>(cap);
    cudaMemcpyAsync(ctx->row_ptr, nrp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s);
    cudaFreeAsync(nrp, s);
    cudaFreeAsync(B.base, s);
    ctx->m = new_m;
    ctx->stats.n_edges = new_m;
    ctx->stats.updates_applied += nops;
    if ((e = cudaGetLastError())) return cuda_error(ctx, e, "apply update batch");
    return BISIM_OK;
}

// The same batch applied to the row store: rows are edited in place, so the
// cost follows the rows the batch touches. Order: copies of every key present
// before the batch, the fold, deletion of the removed copies, deleted and
// revived vertices, then the added copies (rows that run out of room move to
// the pool's tail first). The CSR is left stale.
bisim_status apply_ops_to_store(bisim_ctx* ctx, const bisim_op* d_ops, int64_t nops, uint8_t* vchanged,
                                uint8_t* rowchg, uint8_t* killed, cudaStream_t s) {
    const int32_t n = ctx->n;
    const size_t nn = static_cast<size_t>(std::max(n, 1)) + 1;
    const size_t nb = static_cast<size_t>(std::max<int64_t>(nops, 1));
    cudaError_t e;
    bisim_status st;
    // extra scratch: revived and alive0 flags, two task lists of nops rows per tier,
    // touched rows and their moves (out and in), counters
    size_t extra = 0;
    auto need = [&](size_t b) { extra += (b + 255) & ~size_t(255); };
    need(nn); need(nn);
    need(3 * sizeof(RowTask) * nb); need(3 * sizeof(RowTask) * nb);
    need(4 * nb); need(4 * nb); need(sizeof(RowMove) * nb); need(sizeof(RowMove) * nb);
    need(64);
    Batch B;
    uint8_t* revived = nullptr;
    uint8_t* alive0 = nullptr;
    {
        // the flags are carved first, before batch_begin needs them: allocate them separately
        if ((e = cudaMallocAsync(reinterpret_cast<void**>(&revived), 2 * nn, s))) return cuda_error(ctx, e, "alloc update flags");
        alive0 = revived + nn;
        cudaMemsetAsync(revived, 0, nn, s);
    }
    if ((st = batch_begin(ctx, d_ops, nops, extra, vchanged, killed, revived, alive0, B, s)) != BISIM_OK) {
        cudaFreeAsync(revived, s);
        return st;
    }
    auto done = [&](bisim_status r) {
        cudaFreeAsync(B.base, s);
        cudaFreeAsync(revived, s);
        return r;
    };
    char* scratch = B.extra;
    auto carve = [&](size_t b) { char* p = scratch; scratch += (b + 255) & ~size_t(255); return p; };
    carve(nn);
    carve(nn);
    RowTask* ta = reinterpret_cast<RowTask*>(carve(3 * sizeof(RowTask) * nb));
    RowTask* tb = reinterpret_cast<RowTask*>(carve(3 * sizeof(RowTask) * nb));
    int32_t* touched_o = reinterpret_cast<int32_t*>(carve(4 * nb));
    int32_t* touched_i = reinterpret_cast<int32_t*>(carve(4 * nb));
    RowMove* moves_o = reinterpret_cast<RowMove*>(carve(sizeof(RowMove) * nb));
    RowMove* moves_i = reinterpret_cast<RowMove*>(carve(sizeof(RowMove) * nb));
    unsigned* cnts = reinterpret_cast<unsigned*>(carve(64));     // [0..2] list A, [4..6] list B, [8..9] touched
    TierLists LA{{ta, ta + nb, ta + 2 * nb}, cnts};
    TierLists LB{{tb, tb + nb, tb + 2 * nb}, cnts + 4};
    unsigned* n_touched = cnts + 8;
    const StoreView S{ctx->xro, ctx->xlen, ctx->xcap, ctx->xpe, ctx->yro, ctx->ylen, ctx->ycap, ctx->ype};
    const int64_t nv = B.nv, ne = B.ne;
    KeyTable& T = B.T;
    const int grid = kTierGrid;
    BISIM_SITE(site, "update_rows");

    // copies present before the batch, the fold, and the deletions of copies; each
    // source row a key names is scanned once per pass
    if (ne > 0) {
        Launch L(site, s, 0, 0, 0.0);
        cudaMemsetAsync(cnts, 0, 32, s);
        cudaMemsetAsync(n_touched, 0, 8, s);
        k_mark_kinds<<<grid_for(ne, 256), 256, 0, s>>>(d_ops, B.skp, ne, T);
        k_key_rows<<<grid_for(ne, 256), 256, 0, s>>>(B.keyslot, ne, T, ctx->xmark, ctx->dmark, touched_o, touched_i,
                                                     n_touched);
        k_rows_to_tasks<<<grid, 256, 0, s>>>(touched_i, n_touched + 1, S, ctx->xmark, 0, LB);
        k_rows_to_tasks<<<grid, 256, 0, s>>>(touched_o, n_touched, S, ctx->xmark, 1, LA);
        run_tiers(LB, KeyCountRows{ctx->xpe, alive0, ctx->dmark, T}, s);
    }
    fold_keys(B, killed, rowchg, s);
    if (ne > 0) {
        run_tiers(LA, KeyRemoveRows{ctx->xpe, ctx->dmark, T}, s, false);
        k_remove_long<<<kTierGrid, kTierThreads, 0, s>>>(LA, ctx->xpe, ctx->dmark, T);
        k_clear_dmark<<<grid_for(ne, 256), 256, 0, s>>>(B.keyslot, ne, T, ctx->dmark);
    }
    // deleted and revived vertices
    if (nv > 0) {
        RowTask* pt = tb;
        void* pmem = nullptr;
        int64_t pcap = static_cast<int64_t>(nb);
        if (B.vadds > 0) {
            // revived vertices: one purge task per entry of their in-rows
            unsigned long long* dneed = reinterpret_cast<unsigned long long*>(cnts + 12);
            cudaMemsetAsync(dneed, 0, 8, s);
            k_vertex_tasks<<<grid_for(nv, 256), 256, 0, s>>>(B.V, killed, revived, S, LA, dneed);
            unsigned long long hneed = 0;
            cudaMemcpyAsync(&hneed, dneed, 8, cudaMemcpyDeviceToHost, s);
            if ((e = cudaStreamSynchronize(s))) return done(cuda_error(ctx, e, "size revival purge"));
            if (static_cast<int64_t>(hneed) > pcap) {
                pcap = static_cast<int64_t>(hneed);
                if ((e = cudaMallocAsync(&pmem, 3 * sizeof(RowTask) * static_cast<size_t>(pcap), s)))
                    return done(cuda_error(ctx, e, "alloc revival purge"));
                pt = static_cast<RowTask*>(pmem);
            }
        }
        const TierLists LP{{pt, pt + pcap, pt + 2 * pcap}, cnts + 4};
        Launch L(site, s, 0, 0, 0.0);
        cudaMemsetAsync(cnts, 0, 32, s);
        k_vertex_tasks<<<grid_for(nv, 256), 256, 0, s>>>(B.V, killed, revived, S, LA, nullptr);
        run_tiers(LA, VertexSources{ctx->ype, killed, revived, rowchg, S, LP}, s);
        run_tiers(LP, PurgeTarget{ctx->xpe}, s);
        k_vertex_rows<<<grid_for(nv, 256), 256, 0, s>>>(B.V, killed, revived, S, rowchg);
        if (pmem) cudaFreeAsync(pmem, s);
    }
    // added copies: rows that cannot take them move first
    for (int attempt = 0;; ++attempt) {
        {
            Launch L(site, s, 0, 0, 0.0);
            cudaMemsetAsync(n_touched, 0, 8, s);
            cudaMemsetAsync(ctx->dtail + 2, 0, 16, s);
            k_add_rows<<<grid, 256, 0, s>>>(B.add, B.counters + 1, ctx->addo, ctx->addi, touched_o, touched_i, n_touched);
            k_plan_rows<<<grid, 256, 0, s>>>(touched_o, n_touched, ctx->addo, ctx->xlen, ctx->xcap, ctx->dtail,
                                             ctx->xpool, ctx->dtail + 2, moves_o);
            k_plan_rows<<<grid, 256, 0, s>>>(touched_i, n_touched + 1, ctx->addi, ctx->ylen, ctx->ycap, ctx->dtail + 1,
                                             ctx->ypool, ctx->dtail + 3, moves_i);
        }
        int64_t tails[4] = {0, 0, 0, 0};       // out / in tails, out / in room asked for
        cudaMemcpyAsync(tails, ctx->dtail, sizeof(tails), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s))) return done(cuda_error(ctx, e, "plan row moves"));
        if (tails[0] <= ctx->xpool && tails[1] <= ctx->ypool) break;
        if (attempt > 0) return done(set_error(ctx, BISIM_ENOMEM, "row store full after a rebuild"));
        // a pool is full: rebuild the store (compacted, with room for these moves) and plan again
        k_clear_rows<<<grid, 256, 0, s>>>(touched_o, n_touched, ctx->addo);
        k_clear_rows<<<grid, 256, 0, s>>>(touched_i, n_touched + 1, ctx->addi);
        ctx->csr_stale = true;
        if ((st = store_build(ctx, s, 2 * tails[2], 2 * tails[3])) != BISIM_OK) return done(st);
    }
    {
        const StoreView S2{ctx->xro, ctx->xlen, ctx->xcap, ctx->xpe, ctx->yro, ctx->ylen, ctx->ycap, ctx->ype};
        Launch L(site, s, 0, 0, 0.0);
        cudaMemsetAsync(cnts, 0, 32, s);
        k_move_tasks<<<grid, 256, 0, s>>>(touched_o, n_touched, moves_o, ctx->xro, ctx->xlen, LA);
        k_move_tasks<<<grid, 256, 0, s>>>(touched_i, n_touched + 1, moves_i, ctx->yro, ctx->ylen, LB);
        run_tiers(LA, MoveOut{ctx->xpe, ctx->alive, moves_o}, s);
        run_tiers(LB, MoveIn{ctx->ype, ctx->alive, moves_i}, s);
        k_finish_moves<<<grid, 256, 0, s>>>(touched_o, n_touched, moves_o, ctx->xro, ctx->xlen, ctx->xcap);
        k_finish_moves<<<grid, 256, 0, s>>>(touched_i, n_touched + 1, moves_i, ctx->yro, ctx->ylen, ctx->ycap);
        k_place_adds_rows<<<grid, 256, 0, s>>>(B.add, B.counters + 1, S2);
        k_clear_rows<<<grid, 256, 0, s>>>(touched_o, n_touched, ctx->addo);
        k_clear_rows<<<grid, 256, 0, s>>>(touched_i, n_touched + 1, ctx->addi);
    }
    ctx->csr_stale = true;
    ctx->stats.updates_applied += nops;
    if ((e = cudaGetLastError())) return done(cuda_error(ctx, e, "apply update batch"));
    return done(BISIM_OK);
}

}  // namespace bisim
