/*
 * bisim.h -- C-ABI of the GB300 k-bisimulation library (libbisim_gb300.so).
 *
 * The library computes the forward k-bisimulation partition of a directed,
 * edge-labelled multigraph with one int32 label per vertex and one per edge:
 * the equivalence of Section 2.5 of arXiv 2111.12493, refined round by round
 * as in Algorithm 4 (Section 3.3.1, "Iterative Parallel Hash-Messaging"), with
 * every hash match confirmed by an exact comparison of the full signatures so
 * that the result is the exact partition and not a probabilistic one.
 *
 * Round i -> i+1 (Algorithm 4: SignalMessages, MergeMessages, Hash; the
 * definition of Section 2.5; the chaining parameterization of Section 2.4.2):
 *   S_i(v)     = { (l, P_i[w]) : (v, w, l) is an out-edge of v }   (a set)
 *   P_{i+1}[v] = smallest u with (P_i[u], S_i(u)) == (P_i[v], S_i(v))
 * P_0 groups vertices by label (the labelled variant of Section 2.5); with all
 * labels equal it is the tautology start of the paper's worked example.
 * Block ids are canonical: the smallest vertex id in the block (for batched
 * graphs: the smallest graph-local id). Deleted vertices read -1.
 *
 * Conventions for every call:
 *  - Vertex ids are int32 in [0, n); edge counts are int64.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Work is enqueued on it; calls that return scalars (rounds, block
 *    counts) synchronise it before returning.
 *  - Input arrays may live in device memory or in host memory (pinned host
 *    memory is copied asynchronously, pageable memory synchronously). The
 *    library copies every input into buffers it owns before the call returns
 *    control of the stream; the caller keeps ownership of its arrays and may
 *    reuse them once the stream has passed that point.
 *  - Output arrays are caller-allocated (device or host memory).
 *  - Errors are reported only by return code; no exception crosses the ABI.
 *    After an error the context keeps its last good state, and
 *    bisim_last_error() describes what went wrong.
 *  - A context is not thread-safe: one caller at a time per context.
 */
#ifndef BISIM_GB300_H
#define BISIM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bisim_ctx bisim_ctx;   /* opaque; owned by the library */

typedef enum {
    BISIM_OK = 0,
    BISIM_EINVAL = 1,    /* invalid argument or malformed graph */
    BISIM_ENOMEM = 2,    /* device allocation failed or the memory budget is exceeded */
    BISIM_ECUDA = 3,     /* a CUDA call failed; see bisim_last_error() */
    BISIM_ESTATE = 4,    /* call not valid in the context's current state */
    BISIM_ETIMEOUT = 5,  /* a bounded device-side loop ran out of iterations */
    BISIM_EADMIT = 6     /* request refused by admission control (serving) */
} bisim_status;

enum { BISIM_FIXPOINT = -1 };

/* Option flags. BISIM_FLAG_L2_PIN: mark the current partition as persisting in
 * L2 during bisim_iterate (an access-policy window on the caller's stream for
 * the duration of the call, removed with the persisting lines reset before
 * returning). Off by default: on the 10M-vertex power-law graph the set-aside
 * slowed the rest of the round more than it sped up the gathers. */
enum { BISIM_FLAG_L2_PIN = 1 };

/* BISIM_FLAG_FULL_RECOMPUTE: apply_updates recomputes all k_incremental
 * rounds of the edited graph from scratch instead of maintaining the
 * partition incrementally (same result; the reference point for latency). */
enum { BISIM_FLAG_FULL_RECOMPUTE = 2 };

/* BISIM_FLAG_EAGER: run the rounds of bisim_iterate as host-driven launch
 * sequences, one round at a time. By default the round loop is one captured
 * CUDA graph whose while node repeats a round until the block count stops
 * changing or the round limit is reached, decided on the device; rounds also
 * run eagerly while launch profiling (bisim_profile_enable) is on. */
enum { BISIM_FLAG_EAGER = 4 };

/* BISIM_FLAG_UNION_ROUNDS: batched contexts run the rounds of the disjoint
 * union through the single-graph round kernels for every graph, whatever
 * batch_split says (same partition). Otherwise bisim_iterate on a batched
 * context launches a persistent kernel whose CTAs take the graphs of at most
 * batch_split vertices from a work queue, largest first, and run each graph's
 * rounds, renumbering and collision levels to the end, while the larger graphs
 * go through the union's round kernels at the same time. */
enum { BISIM_FLAG_UNION_ROUNDS = 8 };

/* Direction of the edges that make up a vertex's signature (Section 2.5:
 * forward bisimulation compares outgoing edges, backward bisimulation incoming
 * ones; the forward-backward variant compares both, an out-pair never equal to
 * an in-pair). BISIM_DIR_BOTH needs every edge label in [-2^30, 2^30). */
enum { BISIM_DIR_FORWARD = 0, BISIM_DIR_BACKWARD = 1, BISIM_DIR_BOTH = 2 };

/* Update operations (Section 3.2, incremental summarization of evolving graphs:
 * additions, deletions and modifications of vertices and edges). */
enum {
    BISIM_OP_EDGE_ADD = 0,    /* add edge (src -> dst, label); both endpoints must be live */
    BISIM_OP_EDGE_DEL = 1,    /* remove one edge (src -> dst, label); a no-op if none exists */
    BISIM_OP_VERTEX_ADD = 2,  /* make vertex src live with vertex label `label` (relabels a live one) */
    BISIM_OP_VERTEX_DEL = 3   /* remove vertex src and every edge incident to it */
};

typedef struct {
    int32_t kind;
    int32_t src;
    int32_t dst;
    int32_t label;
} bisim_op;

typedef struct {
    int32_t k_incremental;     /* rounds maintained by apply_updates (default 2) */
    int32_t hash_bits;         /* signature hash width, 1..64 (default 64). Lower values force
                                  collisions and exist to test the exact check; results are
                                  identical at every width, only slower. */
    int32_t small_max_degree;  /* out-degree <= this: one thread per vertex (default 32, max 32) */
    int32_t mid_max_degree;    /* out-degree <= this: one warp (up to 256) or one CTA per vertex,
                                  pair values deduplicated in a shared-memory set (default 8192,
                                  max 8192); above it: hub path, the row cut into chunks over many
                                  CTAs, which insert their pair values into a per-hub table in
                                  device memory (two slots per row entry) behind a small
                                  shared-memory filter */
    int32_t hub_chunk;         /* edges per CTA on the hub path (default 4096, 256..4096) */
    int32_t flags;             /* BISIM_FLAG_* bits (default 0) */
    int64_t mem_budget_bytes;  /* refuse (BISIM_ENOMEM) contexts whose device footprint would
                                  exceed this; 0 = no limit */
    int32_t direction;         /* BISIM_DIR_* (default BISIM_DIR_FORWARD) */
    int32_t n_label_filter;    /* > 0: only edges whose label is one of label_filter[0 .. n)
                                  take part (the label-parameterized edge relation of Section
                                  2.4.2); update operations on other labels are ignored.
                                  0 (default): every edge */
    const int32_t* label_filter;  /* host or device memory, read while the context is created */
    int32_t batch_split;       /* batched contexts: graphs of at most this many vertices are refined
                                  by the persistent kernel, larger ones by the union's round kernels
                                  on the caller's stream while the persistent kernel runs beside
                                  them on a stream of its own (0, the default: every graph through
                                  the round kernels, the fastest split measured on the 4096-graph
                                  workload; INT32_MAX: every graph through the persistent kernel;
                                  bisim_autotune picks it per context). Same partitions either way. */
} bisim_options;

typedef struct {
    int32_t n_vertices;
    int32_t n_graphs;
    int64_t n_edges;
    int32_t rounds;            /* result of the last bisim_iterate (k or the fixpoint round) */
    int32_t rounds_executed;   /* refinement rounds computed by the last bisim_iterate */
    int64_t num_blocks;        /* blocks of the current partition */
    int64_t collision_levels;  /* extra exact-resolution passes taken after hash collisions */
    int64_t device_bytes;      /* device memory held by the context */
    int64_t n_small, n_mid, n_hub;  /* vertices per degree bucket */
    int64_t updates_applied;   /* operations applied by apply_updates so far */
    int64_t last_frontier;     /* vertices recomputed by the last apply_updates */
    int64_t state_builds;      /* full builds of the incremental state: the first one, and one
                                  whenever a level's block ids or index slots could run out in
                                  the next batch (ids of blocks left without members are reused,
                                  so this happens only when the index fills with tombstones) */
} bisim_stats;

/* Fills `opt` with the defaults listed above. */
void bisim_default_options(bisim_options* opt);

/*
 * summarize_init -- create a context from an out-CSR graph (the initialization
 * step of Algorithm 4: every vertex gets its initial id from its label).
 *   n_vertices  number of vertices n >= 0
 *   n_edges     number of edges m >= 0
 *   row_ptr     int64[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = m
 *   col         int32[m], edge targets in [0, n), row v holds the out-edges of v
 *   edge_label  int32[m], any int32 values
 *   vertex_label int32[n], any int32 values (-1 is an ordinary label)
 *   alive       uint8[n] or NULL (all live); a dead vertex may not have edges
 *   opt         options or NULL for defaults
 * Returns BISIM_EINVAL for malformed input (nothing is allocated then).
 * The partition starts at P_0; call bisim_iterate to refine it.
 */
bisim_status summarize_init(bisim_ctx** out, int32_t n_vertices, int64_t n_edges,
                            const int64_t* row_ptr, const int32_t* col,
                            const int32_t* edge_label, const int32_t* vertex_label,
                            const uint8_t* alive, const bisim_options* opt, void* stream);

/*
 * summarize_init_coo -- as summarize_init, from an edge list: src/dst int32[m]
 * in [0, n), edge_label int32[m], in any order (a list sorted by src is
 * detected and placed without atomics). The rows are built on the device,
 * keeping each source's edges in list order. When all three edge arrays are in
 * host memory they are copied in on a stream of the context's own while P_0
 * and the sources' part of the build run on `stream`; such copies of
 * different contexts (calls from several host threads) take turns, one
 * context's edge arrays at a time over the host link.
 */
bisim_status summarize_init_coo(bisim_ctx** out, int32_t n_vertices, int64_t n_edges,
                                const int32_t* src, const int32_t* dst,
                                const int32_t* edge_label, const int32_t* vertex_label,
                                const uint8_t* alive, const bisim_options* opt, void* stream);

/*
 * summarize_init_batched -- many independent graphs refined together as one
 * disjoint union. vertex_offsets / edge_offsets are int64[n_graphs+1] prefix
 * sums; src_local / dst_local are graph-local ids (0 <= id < n_g) of the edges
 * of each graph, stored graph after graph; edge_label int32[total edges];
 * vertex_label int32[total vertices]. No block ever crosses two graphs, and
 * get_partition returns graph-local canonical ids. The result for every graph
 * equals refining that graph alone. bisim_iterate on such a context launches
 * a persistent kernel whose CTAs take the graphs of at most
 * opt->batch_split vertices from a device queue (largest first), each
 * running one graph's rounds, renumbering and collision levels to the end,
 * while the larger graphs go through the union's round kernels on the
 * caller's stream; out_rounds is the largest fixpoint round over the graphs
 * (k for a fixed k) and out_num_blocks the sum of their block counts, as for
 * the union refined as one graph. The per-graph table regions need
 * fewer than 2^32 slots in total, else the union's round kernels run instead
 * (as with BISIM_FLAG_UNION_ROUNDS). apply_updates is not supported on
 * batched contexts (BISIM_ESTATE).
 */
bisim_status summarize_init_batched(bisim_ctx** out, int32_t n_graphs,
                                    const int64_t* vertex_offsets, const int64_t* edge_offsets,
                                    const int32_t* src_local, const int32_t* dst_local,
                                    const int32_t* edge_label, const int32_t* vertex_label,
                                    const bisim_options* opt, void* stream);

/*
 * bisim_iterate -- reset to P_0 and refine (Algorithm 4's k signal phases).
 *   k >= 0          run k rounds (k = 0 leaves the label partition)
 *   k = BISIM_FIXPOINT  run until a round changes nothing, at most `cap` rounds
 *   out_rounds      k, or the fixpoint round r (the first r with P_{r+1} = P_r;
 *                   cap if the cap was hit first); may be NULL
 *   out_num_blocks  number of blocks of the result; may be NULL
 * A round whose block count equals the previous one proves the fixpoint (each
 * round refines the previous partition), so later rounds are skipped; the
 * result is the same partition. Synchronises `stream`.
 */
bisim_status bisim_iterate(bisim_ctx* ctx, int32_t k, int32_t cap, int32_t* out_rounds,
                           int64_t* out_num_blocks, void* stream);

/*
 * apply_updates -- apply a batch of update operations (bisim_op[n_ops]) in
 * array order and bring the partition up to date at k = opt.k_incremental
 * rounds, recomputing only vertices within k reverse hops of a change. By
 * Theorem 2 (Section 3.2.2) the result equals a batch run on the edited graph.
 * A batch naming an out-of-range vertex, a dead endpoint of EDGE_ADD, or an
 * unknown kind is rejected whole with BISIM_EINVAL and nothing changes.
 * Synchronises `stream`.
 */
bisim_status apply_updates(bisim_ctx* ctx, const bisim_op* ops, int64_t n_ops, void* stream);

/*
 * get_partition -- write the current canonical block ids to `block`
 * (int32[n], or int32[total vertices] for batched contexts; -1 for dead
 * vertices).
 */
bisim_status get_partition(bisim_ctx* ctx, int32_t* block, void* stream);

/*
 * get_block_sizes -- the count payload of the summary (Section 3.1: the payload
 * of a vertex summary counts the vertices it summarizes; merging summaries adds
 * the counts): sizes[b] = number of vertices whose block id is b, 0 for every b
 * that is not a block id (dead vertices belong to no block).
 *   sizes  int32[n] output, device or host memory (batched contexts: int32[total
 *          vertices], indexed by the union's vertex id; the block with
 *          graph-local id b of graph g is entry vertex_offsets[g] + b)
 * Synchronises `stream`.
 */
bisim_status get_block_sizes(bisim_ctx* ctx, int32_t* sizes, void* stream);

/*
 * get_summary_edges -- the edges of the summary graph (Section 2.6: one vertex
 * per block, an edge labelled l from the block of u to the block of w for every
 * edge (u, w) with label l of the data graph, parallel edges of one label
 * between two blocks collapsed into one): the distinct triples
 * (P[u], l, P[w]) over the live edges, in lexicographic order of (source
 * block, label as a signed int32, target block). Block ids are those of
 * get_partition, except that batched contexts report the union's vertex ids
 * (the block's smallest vertex over the union).
 *   src_block, label, dst_block  int32[capacity] outputs, device or host memory;
 *                                may be NULL when capacity is 0
 *   capacity   entries the outputs hold; min(capacity, count) are written
 *   out_count  the number of distinct triples (call with capacity 0 to size
 *              the outputs)
 * Uses about 36 bytes of temporary device memory per edge. Synchronises `stream`.
 */
bisim_status get_summary_edges(bisim_ctx* ctx, int32_t* src_block, int32_t* label, int32_t* dst_block,
                               int64_t capacity, int64_t* out_count, void* stream);

/*
 * bisim_autotune -- choose the degree-class thresholds of the round layout
 * of the single-graph round kernels (mid_max_degree: rows above it take the
 * hub path; small_max_degree: rows up to it take one thread each) and the hub
 * chunk size for this context's graph by timing `rounds` refinement rounds
 * (1..64) under each candidate value, one setting at a time, on `stream`; on
 * a batched context then batch_split (which graphs the persistent kernel
 * takes and which the round kernels beside it), each candidate timed as a
 * whole bisim_iterate of `rounds` rounds. The persistent kernel's own tiers
 * are fixed. The chosen values stay in the context (and are written to *out
 * when out is not NULL) and take effect from the next bisim_iterate or
 * apply_updates. Results never depend on these settings. Leaves the
 * context's partition undefined until the next bisim_iterate. Synchronises
 * `stream`.
 */
bisim_status bisim_autotune(bisim_ctx* ctx, int32_t rounds, bisim_options* out, void* stream);

/*
 * bisim_retune -- set a context's tuning options without timing anything:
 * small_max_degree, mid_max_degree, hub_chunk and batch_split are taken from
 * *opt (clamped as at creation); every other field of *opt is ignored. For
 * settings that bisim_autotune chose earlier on a graph of the same shape.
 * Results never depend on them; the round layout is rebuilt with them by the
 * next bisim_iterate or apply_updates (the vertex-ordered CSR it is rebuilt
 * from is made on `stream` first when the context has none). BISIM_EINVAL for
 * a NULL ctx or opt. Synchronises `stream`.
 */
bisim_status bisim_retune(bisim_ctx* ctx, const bisim_options* opt, void* stream);

/*
 * bisim_refine_round_noalloc -- one refinement round (block_in -> block_out)
 * that allocates no memory at all. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory, such as a
 * plugin running inside another runtime that owns the whole device heap (a
 * database's user-defined function, a custom operator of an inference
 * server), or a latency-critical loop that reserves every buffer up front
 * because an allocation may synchronise the device or fail under
 * fragmentation.
 *   row_ptr, col, edge_label  a device-resident out-CSR as in summarize_init
 *                             (every vertex live)
 *   block_in   int32[n] device array: any labelling of the vertices -- the raw
 *              vertex labels for the first round, then the previous output
 *   block_out  int32[n] device array, distinct from block_in: the canonical
 *              ids (smallest vertex of each block) of the partition that keeps
 *              u and v together iff block_in[u] = block_in[v] and their sets of
 *              (edge label, block_in of target) pairs are equal
 *   out_num_blocks  number of blocks of block_out; may be NULL
 * Limits: at most 65536 vertices, 1048576 edges and out-degree 8192; larger
 * graphs, host pointers or block_in == block_out return BISIM_EINVAL and
 * touch nothing. All scratch lives in one fixed array of about 10.5 MB inside
 * the library, which every GPU that loads the library holds until the process
 * exits. The first call on a device looks up that array's device address
 * (once per device). Every call shares the array and clears what it needs at its start, so calls that
 * overlap on the GPU -- from two threads or two streams at once -- race and
 * must be serialised by the caller. Synchronises `stream`.
 */
bisim_status bisim_refine_round_noalloc(int32_t n_vertices, int64_t n_edges, const int64_t* row_ptr,
                                        const int32_t* col, const int32_t* edge_label,
                                        const int32_t* block_in, int32_t* block_out,
                                        int64_t* out_num_blocks, void* stream);

/*
 * bisim_literal_alg4 -- diagnostic: the partition Algorithm 4 (Section 3.3.1)
 * computes when taken literally, with exact identifiers (no hash collisions).
 * Algorithm 4 keeps two identifiers per vertex: id_s is refined like the
 * definition of Section 2.5 in rounds 1 .. k-1; id_o has no own term, takes
 * (edge label, neighbour's id_o) in its first round and only the neighbours'
 * id_o after that; the final round combines the own id_s with the set of the
 * neighbours' id_o and no edge labels. A vertex without out-edges keeps both
 * identifiers. The definition's P_k (bisim_iterate) always refines this
 * partition; where it is strictly finer, the literal algorithm merges classes
 * that the definition separates. Writes canonical ids to block (int32[n],
 * device or host) and the block count to *out_num_blocks (may be NULL).
 * Leaves the context's own partition unchanged. Not for batched contexts
 * (BISIM_ESTATE). Allocates about 2k temporary contexts on an auxiliary graph
 * of 2n vertices; a diagnostic, not a fast path. Synchronises `stream`.
 */
bisim_status bisim_literal_alg4(bisim_ctx* ctx, int32_t k, int32_t* block, int64_t* out_num_blocks,
                                void* stream);

/*
 * bisim_export_state -- the context's state as one self-contained byte blob:
 * the options (direction, label filter, k_incremental, ...), vertex labels and
 * live flags, the current partition, the graph as it stands after every
 * update batch (as an out-CSR of the context's own edge list), and, once
 * apply_updates has built it, the incremental state of Section 3.2 (per level
 * the block of every vertex, the block records and the signature index that
 * play the role of the vertex hash index of Section 3.2.1). Batches applied to
 * an imported context continue exactly where the exported one stood; by
 * Theorem 2 (Section 3.2.2) the partition then equals a batch run on the
 * edited graph.
 *   buf        host memory of `capacity` bytes, or NULL
 *   out_bytes  the blob's size; the blob is written only when capacity >= it
 *              (call with capacity 0 to size the buffer)
 * Not for batched contexts (BISIM_ESTATE). The format is this library's own
 * (versioned, host byte order). Synchronises `stream`.
 */
bisim_status bisim_export_state(bisim_ctx* ctx, void* buf, int64_t capacity, int64_t* out_bytes, void* stream);

/*
 * bisim_import_state -- a new context from a blob of bisim_export_state (host
 * memory, `bytes` long). The graph, options, partition and incremental state
 * are restored as exported, nothing is recomputed but the round layout and
 * the row store of the graph. BISIM_EINVAL for a blob that is not one
 * (magic, version, length or header inconsistent); nothing is allocated then.
 * Synchronises `stream`.
 */
bisim_status bisim_import_state(bisim_ctx** out, const void* buf, int64_t bytes, void* stream);

/* Counters of the context (see bisim_stats). Synchronises nothing. */
bisim_status bisim_get_stats(const bisim_ctx* ctx, bisim_stats* out);

/* Free every device buffer of the context, in the order of the stream its
 * last call used, and wait for that stream (so that the memory pool can hand
 * the memory to the next context at once). NULL is accepted. */
bisim_status summarize_destroy(bisim_ctx* ctx);

/*
 * Kernel timing (process-wide, off by default). When enabled, every kernel the
 * library launches is bracketed by CUDA events on the stream it runs on, and
 * its duration is accumulated per launch site together with the algorithmic
 * bytes the launch had to move (per-unit figures x units processed). Enabling
 * adds two event records per launch; the numbers are read back with
 * bisim_profile_read, which synchronises the recorded events.
 */
typedef struct {
    char name[40];           /* launch site, e.g. "sig_small_4", "verify" */
    int64_t launches;
    double total_ms;         /* summed event-timed durations */
    double alg_bytes;        /* summed algorithmic bytes */
    int64_t vertices;        /* vertices processed */
    int64_t edges;           /* edges processed */
} bisim_kernel_profile;

void bisim_profile_enable(int32_t enable);
void bisim_profile_reset(void);
/* Copies up to `max` entries into `out` and returns how many sites exist. */
int32_t bisim_profile_read(bisim_kernel_profile* out, int32_t max);
/* Kernels launched by this library in this process so far (always counted). */
int64_t bisim_launch_count(void);

/* Description of the last error on ctx, or of the calling thread's last
 * failed call when ctx is NULL. Never NULL. */
const char* bisim_last_error(const bisim_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* BISIM_GB300_H */
