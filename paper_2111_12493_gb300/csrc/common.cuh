// Internal declarations shared by the translation units of libbisim_gb300.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "bisim.h"

namespace bisim {

// ----------------------------------------------------------------------------- constants

constexpr int kSmallClasses = 4;          // thread-per-vertex classes: D = 4, 8, 16, 32
constexpr int kMidClasses = 8;            // CTA-per-vertex classes: N = 64 .. 8192
constexpr int kMidMaxN = 8192;            // largest CTA-path key count (64 KB of shared memory)
constexpr int kHubChunkMax = 4096;        // hub-path edges per CTA
constexpr int kMaxIncLevels = 16;         // largest k_incremental
constexpr int kClassHub = kSmallClasses + kMidClasses;   // 12
constexpr int kNumClasses = kClassHub + 1;               // 13
constexpr uint8_t kClassDead = 255;

// Degree classes of the dense round layout (all live vertices every round):
//   0..6   one thread per vertex for out-degree 0, 1, 2, 3-4, 5-8, 9-16, 17-32
//   7..9   one warp per vertex, shared-memory set of 2N slots, N = 64, 128, 256
//   10..14 one CTA per vertex, N = 512 .. 8192
//   15     hubs: rows cut into chunks over many CTAs, values deduplicated by bucket
constexpr int kDWarp0 = 7;
constexpr int kDMid0 = 10;
constexpr int kDHub = 15;
constexpr int kDClasses = 16;
constexpr uint32_t kDDead = 16;           // dead vertices sort after every class

constexpr uint64_t kSaltKey = 0x243f6a8885a308d3ull;     // per-pair key -> m value
constexpr uint64_t kSaltSig = 0x13198a2e03707344ull;     // own term of the signature hash
constexpr uint64_t kSaltLabel = 0xa4093822299f31d0ull;   // label partition hash
constexpr uint64_t kLevelStep = 0x9e3779b97f4a7c15ull;   // re-hash step of collision levels

// device error bits
constexpr unsigned kErrTableFull = 1u;
constexpr unsigned kErrHubFull = 2u;
constexpr unsigned kErrBadInput = 4u;

// ----------------------------------------------------------------------------- hashing

// SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014). A bijection on 64-bit words.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// The value stored for one (edge label, neighbour block) pair. mix64 is a
// bijection, so a set of these values identifies the set of pairs exactly;
// lists are kept sorted by this value, which gives every path the same
// canonical order.
__device__ __forceinline__ uint64_t pair_value(int32_t label, int32_t block) {
    uint64_t key = (static_cast<uint64_t>(static_cast<uint32_t>(label)) << 32) |
                   static_cast<uint32_t>(block);
    return mix64(key ^ kSaltKey);
}

// Order-independent 64-bit hash of a signature (own block p, set S given by
// its size c and the wrap-around sum of its pair values). Algorithm 4's Hash
// is order independent too; the own block plays the role of its (self, id) tuple.
__device__ __forceinline__ uint64_t sig_hash(int32_t p, uint32_t c, uint64_t sum) {
    uint64_t h = mix64(((static_cast<uint64_t>(static_cast<uint32_t>(p)) << 32) | c) ^ kSaltSig);
    return mix64(h + sum);
}

__device__ __forceinline__ uint64_t label_hash(int32_t g, int32_t label) {
    uint64_t key = (static_cast<uint64_t>(static_cast<uint32_t>(g)) << 32) |
                   static_cast<uint32_t>(label);
    return mix64(key ^ kSaltLabel);
}

__device__ __forceinline__ uint64_t level_hash(uint64_t h0, uint32_t level, uint64_t hmask) {
    uint64_t h = level == 0 ? h0 : mix64(h0 ^ (kLevelStep * level));
    return h & hmask;
}

// Signature of one position of the dense rounds: the hash of (own block, |S|,
// pair values), |S| and the own block P_i[v], in one 16-byte record, so that
// the verification reads one sector per side to compare two of them.
struct __align__(16) SigRec {
    unsigned long long hash;
    int32_t cnt;
    int32_t own;
};

// ----------------------------------------------------------------------------- signature table

// One 8-byte slot of the open-addressing signature table:
//   bits 63..36  fingerprint: the top 28 bits of the signature hash
//   bits 35..32  epoch 1..15; a slot whose epoch is not the current one is free,
//                so the table needs clearing only when the epoch wraps
//   bits 31..0   the smallest vertex inserted with this fingerprint this epoch
// Two different signatures that meet in one slot with equal fingerprints are
// merged here and split again by the exact verification pass.
struct __align__(8) Slot {
    unsigned long long w;
};

constexpr unsigned long long kSlotEpochMask = 0xf00000000ull;
constexpr unsigned long long kSlotKeyMask = ~0xffffffffull;     // fingerprint | epoch
constexpr uint32_t kEpochCycle = 15;

struct TableRef {
    Slot* slots;
    uint64_t mask;        // nslots - 1
    uint64_t epoch;       // 1..15, already shifted into bits 32..35
    uint64_t hmask;       // hash width mask (tests only narrow it)
};

struct DevState {
    unsigned long long blocks;      // vertices that are the minimum of their block
    unsigned int unresolved;        // vertices pushed to the next collision level
    unsigned int error;             // kErr* bits
    unsigned long long aux;         // dense rounds: row words read by the exact set comparisons
    unsigned int deferred;          // vertices whose set comparison is left to k_verify_deferred
    unsigned int pairs;             // dense rounds: small pairs left to a warp comparison
    unsigned int listed;            // dense rounds: positions that need the table this round
    unsigned int unsorted;          // COO build: some edge's source is smaller than the one before it
};

__device__ __forceinline__ unsigned long long table_read(const TableRef& t, uint64_t pos) {
    return *reinterpret_cast<volatile unsigned long long*>(&t.slots[pos].w);
}

// Insert `h` (already masked) for vertex v into the region [base, base + mask]
// of the table (mask + 1 a power of two; probing wraps inside the region);
// returns the slot index or ~0u on overflow. `first` is the word already read
// from the home slot base + (h & mask) (callers issue that read early to
// overlap it with other work).
__device__ __forceinline__ uint32_t table_insert_at(const TableRef& t, uint64_t h, int32_t v, uint64_t base,
                                                    uint64_t mask, unsigned long long first, unsigned* err) {
    const unsigned long long tag = (h & ~0xfffffffffull) | t.epoch;
    const unsigned long long want = tag | static_cast<uint32_t>(v);
    uint64_t off = h & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        const uint64_t pos = base + off;
        unsigned long long cur = probe == 0 ? first : table_read(t, pos);
        for (;;) {
            if ((cur & kSlotEpochMask) != t.epoch) {            // free in this epoch: claim it
                const unsigned long long prev = atomicCAS(&t.slots[pos].w, cur, want);
                if (prev == cur) return static_cast<uint32_t>(pos);
                cur = prev;
                continue;
            }
            if ((cur & kSlotKeyMask) == tag) {                  // same fingerprint: keep the smaller vertex
                // popular signatures are inserted by many vertices; the plain
                // read above skips the atomic when a smaller one is recorded
                while (static_cast<uint32_t>(v) < static_cast<uint32_t>(cur)) {
                    const unsigned long long prev = atomicCAS(&t.slots[pos].w, cur, want);
                    if (prev == cur) break;
                    cur = prev;
                }
                return static_cast<uint32_t>(pos);
            }
            break;                                               // another signature: probe on
        }
        off = (off + 1) & mask;
    }
    atomicOr(err, kErrTableFull);
    return ~0u;
}

__device__ __forceinline__ uint32_t table_insert_in(const TableRef& t, uint64_t h, int32_t v, uint64_t base,
                                                    uint64_t mask, unsigned* err) {
    return table_insert_at(t, h, v, base, mask, table_read(t, base + (h & mask)), err);
}

// Insert `h` (already masked) for vertex v anywhere in the table.
__device__ __forceinline__ uint32_t table_insert(const TableRef& t, uint64_t h, int32_t v, unsigned* err) {
    return table_insert_in(t, h, v, 0, t.mask, err);
}

__device__ __forceinline__ int32_t table_rep(const Slot* slots, uint32_t pos) {
    return static_cast<int32_t>(static_cast<uint32_t>(slots[pos].w));
}

// ----------------------------------------------------------------------------- shared-memory sets

// Inserts pair value mv into a shared-memory open-addressing set (0 = empty;
// the value 0 itself is tracked by *zero). Returns true for the first inserter.
__device__ __forceinline__ bool smem_set_insert(unsigned long long* tab, uint32_t mask, unsigned* zero,
                                                unsigned long long mv) {
    if (mv == 0ull) return atomicExch(zero, 1u) == 0u;
    uint32_t pos = static_cast<uint32_t>(mv) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long cur = tab[pos];
        if (cur == mv) return false;
        if (cur == 0ull) {
            const unsigned long long prev = atomicCAS(&tab[pos], 0ull, mv);
            if (prev == 0ull) return true;
            if (prev == mv) return false;
        }
        pos = (pos + 1) & mask;
    }
    return false;   // unreachable: the set has twice as many slots as keys
}

__device__ __forceinline__ bool smem_set_contains(const unsigned long long* tab, uint32_t mask, unsigned zero,
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

// ----------------------------------------------------------------------------- hub tables

// Per-hub dedup table of pair values (0 = empty; the pair value 0 is tracked by a flag).
struct HubChunk {
    int32_t hub;      // index into the hub list
    int32_t vertex;
    int64_t begin;    // edge range [begin, end)
    int64_t end;
};

struct HubAcc {
    unsigned long long sum;
    unsigned int count;
    unsigned int zero;
};

// Degree buckets of a set of vertices: vertices grouped by class (see
// kNumClasses) plus the hub-path layout for the vertices of the hub class.
struct Buckets {
    const int32_t* class_list = nullptr;
    int64_t begin[kNumClasses + 1] = {};
    int64_t edges[kNumClasses] = {};
    const int32_t* hub_list = nullptr;
    int64_t n_hub = 0;
    const HubChunk* chunks = nullptr;
    int64_t n_chunks = 0;
    const int64_t* toff = nullptr;
    const uint32_t* tmask = nullptr;
    unsigned long long* tab = nullptr;
    int64_t tab_words = 0;
    HubAcc* acc = nullptr;
};

// ----------------------------------------------------------------------------- device buffer helper

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace bisim

// ----------------------------------------------------------------------------- context

struct bisim_ctx {
    int32_t n = 0;
    int64_t m = 0;
    int32_t n_graphs = 1;
    bisim_options opt{};
    int device = 0;

    // graph (out-CSR) -- owned
    int64_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    int32_t* elab = nullptr;
    int32_t* vlabel = nullptr;
    uint8_t* alive = nullptr;      // may be null: all live
    int32_t* gid = nullptr;        // batched only
    int64_t* voff = nullptr;       // batched only, [n_graphs+1]

    // partition state
    int32_t* P0 = nullptr;
    int32_t* P[2] = {nullptr, nullptr};
    int cur = 0;                   // P[cur] is the current partition
    int32_t* cnt = nullptr;        // |S_v|
    unsigned long long* skey = nullptr;   // sorted unique pair values, at row_ptr[v]
    uint32_t* slot = nullptr;
    bisim::Slot* table = nullptr;
    uint64_t nslots = 0;
    uint32_t epoch32 = 0;

    // degree buckets
    int32_t* class_list = nullptr;                 // vertices grouped by class
    int64_t class_begin[bisim::kNumClasses + 1] = {};
    int64_t class_edges[bisim::kNumClasses] = {};   // out-edges of the vertices of each class
    int32_t* hub_list = nullptr;                   // = class_list + class_begin[kClassHub]
    int64_t n_hub = 0;
    int64_t* hub_toff = nullptr;                   // table offset per hub (in words)
    uint32_t* hub_tmask = nullptr;                 // table size - 1 per hub
    unsigned long long* hub_tab = nullptr;
    int64_t hub_tab_words = 0;
    bisim::HubChunk* chunks = nullptr;
    int64_t n_chunks = 0;
    bisim::HubAcc* hub_acc = nullptr;

    // dense round layout: live vertices grouped by degree class (then the dead
    // ones), their out-rows copied in that order as packed (label << 32 | target)
    bool dense_ready = false;
    int64_t layout_version = 0;                      // counts the layouts built
    int32_t* dvert = nullptr;                        // [n] position -> vertex
    int32_t* dvpos = nullptr;                        // [n] vertex -> position
    int64_t* dprp = nullptr;                         // [n_live + 1] row offsets into dpe
    unsigned long long* dpe = nullptr;               // [m] packed edges in position order
    int64_t dpe_cap = 0;
    int64_t dbegin[bisim::kDClasses + 1] = {};       // class -> first position; dbegin[kDClasses] = n_live
    int64_t dedge_begin[bisim::kDClasses + 1] = {};  // class -> first packed edge
    bisim::Slot* rtable = nullptr;                   // batched contexts: one table region per graph
    uint64_t n_rslots = 0;
    int64_t* rbase = nullptr;                        // [n_graphs] first slot of the graph's region
    uint32_t* rmask = nullptr;                       // [n_graphs] region size - 1 (a power of two)
    uint32_t* dslot = nullptr;                       // [n] table slot per position
    bisim::SigRec* dsig = nullptr;                   // [n] signature hash, |S| and own block per position
    int2* dpairs = nullptr;                          // [n] (position, representative's position) for a CTA compare
    int2* dsmall = nullptr;                          // [n] the same for rows of at most 32 edges (warp compare)
    uint8_t* djoined = nullptr;                      // [n] by position: another vertex joined this one's block last round
    uint8_t* downs = nullptr;                        // [n] by position: the vertex was its block's id last round
    // active list of the dense rounds: the positions whose vertex is not alone
    // in its block (ascending, hence grouped by degree class); a vertex alone in
    // its block stays alone in every later round, so the list only shrinks
    int32_t* dact = nullptr;                         // [n] active positions
    int32_t* dact2 = nullptr;                        // [n] the next round's list while it is compacted
    int64_t* daoff = nullptr;                        // [kDClasses + 1] class c's entries: dact[daoff[c] .. daoff[c+1])
    int64_t* dtile = nullptr;                        // [tiles + 2 + kDClasses] survivors per tile, then their offsets; the new length; survivors per class
    int64_t n_tiles = 0;                             // tiles of kActTile entries covering all live positions
    unsigned long long* dwork = nullptr;             // launch profiling: signature work counters of a round
    bisim::HubChunk* dchunks = nullptr;              // hub rows cut into chunks of at most 4096 edges
    int64_t n_dchunks = 0;
    int64_t n_dhub = 0;
    unsigned long long* htab = nullptr;              // [2 * hub edges] per-hub open-addressing tables of pair values
    int64_t hub_edges = 0;
    bisim::HubAcc* dacc = nullptr;
    void* round_graph = nullptr;                     // cudaGraphExec_t of the device-side round loop
    void* capture_stream = nullptr;                  // cudaStream_t used only to capture it
    void* copy_stream = nullptr;                     // cudaStream_t bringing a host COO list in beside the build
    void* copy_events[4] = {nullptr, nullptr, nullptr, nullptr};   // buffers ready; sources, targets, labels copied
    void* dloop = nullptr;                           // loop state on the device
    void* hloop = nullptr;                           // its pinned host mirror
    int64_t round_graph_launches = 0;                // kernels in one captured round

    // batched contexts: the persistent per-graph kernel (segment.cu)
    int32_t* seg_order = nullptr;                    // [n_graphs] work queue of the persistent kernel, largest graph first
    std::vector<int64_t> seg_vcount;                 // host: vertices per graph
    std::vector<int32_t> seg_sorted;                 // host: graphs, largest first (by edges, then vertices)
    int32_t seg_split = -1;                          // batch_split the queue and seg_big were built for
    int32_t seg_n_small = 0;                         // graphs in the persistent kernel's queue
    uint8_t* seg_big = nullptr;                      // [n_graphs] the graph runs through the union's round kernels
    bisim::Slot* seg_table = nullptr;                // the persistent kernel's table regions while the union runs beside it
    void* seg_stream = nullptr;                      // cudaStream_t of the persistent kernel beside the union
    void* seg_events[2] = {nullptr, nullptr};        // fork and join of the two streams
    int64_t* seg_e0 = nullptr;                       // [n] first entry of the vertex's row in dpe
    int32_t* seg_deg = nullptr;                      // [n] its length
    int64_t seg_rows_version = -1;                   // layout_version the two arrays were taken from
    unsigned long long* seg_hash = nullptr;          // [n] signature hash by vertex
    uint8_t* seg_own = nullptr;                      // [n] the vertex was its block's id last round
    uint8_t* seg_joined = nullptr;                   // [n] another vertex joined its block last round
    int32_t* seg_lists = nullptr;                    // [4 n] per-graph lists of a round
    void* seg_state = nullptr;                       // device SegState
    void* seg_host = nullptr;                        // its pinned mirror

    // collision resolution
    int32_t* ulist[2] = {nullptr, nullptr};
    int32_t* dlist = nullptr;      // vertices whose verification needs a set comparison
    bisim::DevState* dstate = nullptr;
    bisim::DevState* hstate = nullptr;   // pinned mirror

    // updates
    int32_t* esrc = nullptr;       // source vertex of every CSR edge (kept once updates start)
    int64_t esrc_cap = 0;
    int64_t skey_cap = 0;          // capacity of skey in values
    bool buckets_dirty = false;    // the label partition no longer matches the graph
    int32_t cur_k = 0;             // rounds of the current partition

    // dynamic adjacency of the incremental path (built with its state): out-rows
    // and in-rows with spare capacity in two pools, edited in place by batches;
    // while csr_stale is set, the CSR above lags behind it and is rebuilt from it
    // before any other path reads the graph
    bool store_ready = false;
    bool csr_stale = false;
    int64_t* xro = nullptr;        // [n] out-row offset into xpe
    int32_t* xlen = nullptr;       // [n] entries in use (deleted ones included)
    int32_t* xcap = nullptr;       // [n] capacity
    unsigned long long* xpe = nullptr;   // out-pool: packed (label << 32 | target), ~0 deleted
    int64_t xpool = 0;             // out-pool entries
    int64_t* yro = nullptr;        // [n] in-row offset into ype
    int32_t* ylen = nullptr;
    int32_t* ycap = nullptr;
    int32_t* ype = nullptr;        // in-pool: source vertices
    int64_t ypool = 0;
    int64_t* dtail = nullptr;      // [4] device: out-pool and in-pool tails, room the last plan asked for
    int32_t* addo = nullptr;       // [n] per-batch adds per out-row (kept zero between batches)
    int32_t* addi = nullptr;       // [n] per-batch adds per in-row
    uint32_t* xmark = nullptr;     // [n] per-batch: out-row already listed (kept zero between batches)
    uint32_t* dmark = nullptr;     // [n / 32 + 1] per-batch bitmap: target of a deleted key (kept zero)
    int32_t inc_small_max = 0;     // thread-per-vertex limit of the incremental path's current frontiers

    // incremental maintenance (apply_updates): per level j = 0..inc_k, block ids
    // per vertex, |S| per vertex, block records and a hash index key -> block
    int32_t inc_k = -1;            // levels built (-1: no incremental state)
    int32_t* lid[bisim::kMaxIncLevels + 1] = {};
    uint8_t* lstale[bisim::kMaxIncLevels + 1] = {};  // per vertex: its block at this level has no current index key
    int32_t* lcnt[bisim::kMaxIncLevels + 1] = {};
    unsigned long long* bkey[bisim::kMaxIncLevels + 1] = {};
    int32_t* bcnt[bisim::kMaxIncLevels + 1] = {};
    int32_t* bmin[bisim::kMaxIncLevels + 1] = {};
    unsigned long long* ikey[bisim::kMaxIncLevels + 1] = {};
    int32_t* ibid[bisim::kMaxIncLevels + 1] = {};
    int32_t* lfree[bisim::kMaxIncLevels + 1] = {};  // [bcap] block ids freed by earlier batches, reused first
    int64_t bnext[bisim::kMaxIncLevels + 1] = {};   // next never-used block id
    int64_t nfree[bisim::kMaxIncLevels + 1] = {};   // ids in lfree after the last batch
    long long* lfreec = nullptr;   // device [kMaxIncLevels + 1][3]: ids in lfree, taken, freed (in the scratch)
    int64_t itomb[bisim::kMaxIncLevels + 1] = {};   // tombstones in the index
    void* inc_ws = nullptr;        // per-batch work buffers of the incremental path (kept between batches)
    int64_t bcap = 0;              // block records per level
    uint64_t isize = 0;            // index slots per level (power of two)

    // direction and label filter of the summarized edges (direction.cu)
    int32_t* dfilter = nullptr;    // [nfilter] listed edge labels, sorted, unique
    int32_t nfilter = 0;           // 0: every label

    // bookkeeping
    void* last_stream = nullptr;   // stream of the last call (the context's memory is freed in its order)
    std::vector<void*> allocs;
    int64_t device_bytes = 0;
    bisim_stats stats{};
    int64_t last_blocks = 0;
    std::string err;
};

namespace bisim {

// ----------------------------------------------------------------------------- host helpers (api.cu)

bisim_status set_error(bisim_ctx* ctx, bisim_status st, const std::string& msg);
bisim_status cuda_error(bisim_ctx* ctx, cudaError_t e, const char* what);
cudaError_t ctx_alloc(bisim_ctx* ctx, void** p, size_t bytes, cudaStream_t s);
// 256-byte pinned host blocks from process-lifetime slabs (nullptr if none can be had).
void* pinned_take();
void pinned_give(void* p);

// ----------------------------------------------------------------------------- primitives (sort.cu)

// Exclusive prefix sum of int64 values; `tmp` must hold scan_temp_words(n) words.
size_t scan_temp_words(int64_t n);
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s);

// Stable LSD radix sort of (u32 key, u64 value) pairs on the low `bits` key bits.
// Buffers are ping-ponged; returns 0 if the result ended in (k0, v0), 1 if in (k1, v1).
size_t radix_temp_words(int64_t m);
// `site_name` names the launch-timing sites of the passes ("<name>_hist", "<name>_scatter").
int radix_sort_pairs(uint32_t* k0, uint64_t* v0, uint32_t* k1, uint64_t* v1, int64_t m, int bits,
                     int64_t* tmp, cudaStream_t s, const char* site_name = "radix");

// ----------------------------------------------------------------------------- graph build (graph.cu)

// Events of a COO list being copied in on another stream (sources, targets,
// labels, in that order): build_from_coo waits for each array just before its
// first use.
struct CooArrival {
    cudaEvent_t src, dst, lab;
    // called (when set) as soon as the last array has arrived, before the
    // rows are placed
    void (*arrived)(void*) = nullptr;
    void* arrived_arg = nullptr;
};
bisim_status build_from_coo(bisim_ctx* ctx, const int32_t* src, const int32_t* dst,
                            const int32_t* elab, cudaStream_t s, const CooArrival* arrival = nullptr);
bisim_status build_from_csr(bisim_ctx* ctx, const int64_t* row_ptr, const int32_t* col,
                            const int32_t* elab, cudaStream_t s);


// ----------------------------------------------------------------------------- dynamic adjacency (store.cu)

// Builds the out-/in-row store from the current CSR (all rows with spare
// capacity, and at least room_out / room_in free entries at the pools' tails).
bisim_status store_build(bisim_ctx* ctx, cudaStream_t s, int64_t room_out = 0, int64_t room_in = 0);
void store_release(bisim_ctx* ctx, cudaStream_t s);
// Rebuilds row_ptr / col / elab (and m) from the store when batches edited it.
bisim_status csr_from_store(bisim_ctx* ctx, cudaStream_t s);

// ----------------------------------------------------------------------------- refinement (refine.cu)

bisim_status compute_p0(bisim_ctx* ctx, cudaStream_t s);
// Advances the signature table's epoch (clearing the table when it wraps).
TableRef next_epoch(bisim_ctx* ctx, cudaStream_t s);
bisim_status refine_round(bisim_ctx* ctx, cudaStream_t s, int64_t* out_blocks);
// One signature round over the vertices of `B` (all of them, or the `vcount`
// listed in `vlist` for verification): Pout[v] = smallest listed vertex with
// v's exact signature over the labelling Pin; hout[v] (nullable) receives the
// signature hash that was inserted.
bisim_status signature_round(bisim_ctx* ctx, const Buckets& B, const int32_t* Pin, int32_t* Pout,
                             const int32_t* vlist, int64_t vcount, unsigned long long* hout, cudaStream_t s,
                             int64_t* out_blocks);
Buckets ctx_buckets(const bisim_ctx* ctx);
bisim_status alloc_refine_state(bisim_ctx* ctx, cudaStream_t s);
void pin_partition_in_l2(bisim_ctx* ctx, const int32_t* P, cudaStream_t s);
void unpin_partition(bisim_ctx* ctx, cudaStream_t s);
void launch_local_ids(const bisim_ctx* ctx, int32_t* out, cudaStream_t s);

// ----------------------------------------------------------------------------- updates (update.cu)

void ctx_free(bisim_ctx* ctx, void* p, size_t bytes, cudaStream_t s);
bisim_status ensure_edge_sources(bisim_ctx* ctx, cudaStream_t s);
bisim_status apply_ops_to_graph(bisim_ctx* ctx, const bisim_op* d_ops, int64_t nops, uint8_t* vchanged,
                                uint8_t* rowchg, uint8_t* killed, cudaStream_t s);
// The same batch applied in place to the row store (the CSR becomes stale).
bisim_status apply_ops_to_store(bisim_ctx* ctx, const bisim_op* d_ops, int64_t nops, uint8_t* vchanged,
                                uint8_t* rowchg, uint8_t* killed, cudaStream_t s);

// ----------------------------------------------------------------------------- rounds (api.cu)

// allow_graph: the loop may run as the captured graph (callers that rebuild the
// layout for every call, like the full recompute of an update batch, pass false).
bisim_status run_rounds(bisim_ctx* ctx, int32_t k, int32_t cap, cudaStream_t s, int32_t* out_rounds,
                        int32_t* out_executed, int64_t* out_blocks, bool allow_graph = true);
// The two halves of the dense path of run_rounds: reset to P_0 and list the
// positions (only those of the graphs with keep_graph[g] != 0 when given),
// then refine from there; out_prev / prev is |P_0| as the rounds count it,
// out_dropped the live vertices left out (counted as blocks by the rounds).
bisim_status dense_rounds_begin(bisim_ctx* ctx, cudaStream_t s, const uint8_t* keep_graph, int64_t* out_prev,
                                int64_t* out_dropped);
bisim_status dense_rounds_run(bisim_ctx* ctx, int32_t k, int32_t cap, cudaStream_t s, int64_t prev,
                              int32_t* out_rounds, int32_t* out_executed, int64_t* out_blocks, bool allow_graph);
bisim_status refresh_after_edit(bisim_ctx* ctx, cudaStream_t s);

// ----------------------------------------------------------------------------- dense rounds (dense.cu)

// Builds (or rebuilds after an edit) the dense round layout of the current CSR.
bisim_status dense_prepare(bisim_ctx* ctx, cudaStream_t s);
// The layout's positions, classes and row offsets from the out-degrees (deg[n]).
bisim_status dense_layout_positions(bisim_ctx* ctx, const int32_t* deg, cudaStream_t s);
// Batched contexts: drops from the active list the positions of the graphs
// with keep_graph[g] == 0 (marked alone, so no round kernel touches them) and
// turns *prev from |P_0| into the count the rounds see: P_0's blocks of the
// kept graphs plus the dropped live vertices (k_round_begin counts every
// unlisted live vertex as a block).
bisim_status dense_keep_graphs(bisim_ctx* ctx, cudaStream_t s, const uint8_t* keep_graph, int64_t* prev,
                               int64_t* dropped);
// The hub part of the layout, after the packed rows exist (or, with
// pack_from_csr, copying the hub rows from the vertex-ordered CSR); marks the
// layout ready.
bisim_status dense_layout_hubs(bisim_ctx* ctx, bool pack_from_csr, cudaStream_t s);
// Batched contexts: one signature-table region per graph (sized for the graph,
// load <= 0.6), so that the inserts of a graph's vertices stay in a small span.
bisim_status dense_region_table(bisim_ctx* ctx, const int64_t* voff_host, int32_t n_graphs, cudaStream_t s);

// ----------------------------------------------------------------------------- batched rounds (segment.cu)

// Uploads the work queue of the persistent batched kernel (graphs by size, largest first).
bisim_status segment_init(bisim_ctx* ctx, const int64_t* voff_host, const int64_t* eoff_host, int32_t n_graphs,
                          cudaStream_t s);
// Whether bisim_iterate runs the persistent per-graph kernel for this context.
bool segment_usable(const bisim_ctx* ctx);
void segment_release(bisim_ctx* ctx);
// All rounds of every graph of a batched context in one launch; the partition ends in P[0].
bisim_status segment_rounds(bisim_ctx* ctx, int32_t k, int32_t cap, cudaStream_t s, int32_t* out_rounds,
                            int32_t* out_executed, int64_t* out_blocks);
// The vertex-ordered CSR (row_ptr, col, elab), rebuilt from the layout when a
// context was built straight into it (updates and list-mode paths need it).
bisim_status ensure_vertex_csr(bisim_ctx* ctx, cudaStream_t s);
// Writes -1 for the dead vertices into both partition buffers.
void dense_mark_dead(bisim_ctx* ctx, cudaStream_t s);
// Prepares a run of rounds from P_0: dead vertices, and no block known to be a singleton.
void dense_start(bisim_ctx* ctx, cudaStream_t s);
// One refinement round P[cur] -> P[cur ^ 1] over every live vertex.
bisim_status dense_round(bisim_ctx* ctx, cudaStream_t s, int64_t* out_blocks);
// Finishes a round stopped by the device-side loop at a hash collision.
bisim_status dense_finish_round(bisim_ctx* ctx, cudaStream_t s, int64_t* out_blocks);
struct GraphRounds {
    int32_t executed;     // rounds run on the device
    int32_t rounds;       // r when stop == 1
    int64_t blocks;       // block count after the last round
    int32_t stop;         // 1 done, 2 the last round needs its collision levels, 3 device error
};
// Whether the rounds may run as the captured device-side loop.
bool dense_graph_usable(const bisim_ctx* ctx);
// Runs up to `limit` rounds from P[0] as one graph launch (the loop checks the
// block count on the device); the result is in P[0] unless stop == 2.
bisim_status dense_graph_rounds(bisim_ctx* ctx, cudaStream_t s, int32_t limit, bool fixpoint, int64_t prev_blocks,
                                GraphRounds* out);
// Releases the graph, its capture stream and pinned mirror.
void dense_release(bisim_ctx* ctx);

// ----------------------------------------------------------------------------- direction and label filter (direction.cu)

// An edge list in device memory that the library owns (freed by edge_view_free).
struct EdgeView {
    int32_t* src = nullptr;
    int32_t* dst = nullptr;
    int32_t* lab = nullptr;
    int64_t* eoff = nullptr;       // batched: per-graph offsets of the view's edges [G + 1]
    int64_t m = 0;
};
// Whether the context refines the caller's edges unchanged (forward, no filter).
bool edge_view_identity(const bisim_ctx* ctx);
// Copies the options' label filter (sorted, unique) into the context.
bisim_status edge_view_setup(bisim_ctx* ctx, const bisim_options* opt, cudaStream_t s);
// The internal edge list of the context's direction and filter for device
// arrays (src, dst, lab)[m]; eoff (device, [G + 1]) gives per-graph offsets
// of batched inputs, or is null.
bisim_status edge_view_coo(bisim_ctx* ctx, const int32_t* src, const int32_t* dst, const int32_t* lab, int64_t m,
                           const int64_t* eoff, int32_t G, cudaStream_t s, EdgeView* out);
void edge_view_free(EdgeView* v, cudaStream_t s);
// An update batch mapped onto the internal edge list (device arrays; *out is
// freed by the caller with cudaFreeAsync).
bisim_status edge_view_ops(bisim_ctx* ctx, const bisim_op* ops, int64_t n, cudaStream_t s, bisim_op** out,
                           int64_t* out_n);
// Source vertex of every edge of a CSR (src[m]); a row_ptr that is not a
// prefix sum of [0, m] gives BISIM_EINVAL and writes nothing out of range.
bisim_status csr_sources(bisim_ctx* ctx, const int64_t* row_ptr, int32_t n, int64_t m, int32_t* src, cudaStream_t s);

// ----------------------------------------------------------------------------- incremental levels (inc.cu)

bisim_status inc_build(bisim_ctx* ctx, cudaStream_t s);
// The row store and the levels' arrays of K levels, allocated and not filled (state import).
bisim_status inc_alloc_levels(bisim_ctx* ctx, int K, int64_t bcap, uint64_t isize, cudaStream_t s);
// Sets the next unused block id of every level (host and device counters).
bisim_status inc_set_next_ids(bisim_ctx* ctx, const int64_t* bnext, cudaStream_t s);
bisim_status inc_update(bisim_ctx* ctx, const uint8_t* vchanged, const uint8_t* rowchg, int64_t n_ops,
                        cudaStream_t s);
void inc_release(bisim_ctx* ctx, cudaStream_t s);
bisim_status write_current(bisim_ctx* ctx, cudaStream_t s);

}  // namespace bisim
