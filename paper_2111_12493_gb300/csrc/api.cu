// C-ABI entry points (declared in include/bisim.h): argument checks, input
// staging, context lifetime, and the round loop of bisim_iterate.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <string>

#include "common.cuh"
#include "prof.cuh"

namespace bisim {

namespace {

thread_local std::string g_last_error = "no error";

// Small pinned host blocks (status mirrors of contexts) come from slabs that
// live for the whole process: allocating and freeing pinned memory per
// context costs far more than the context's own work on small graphs, and
// freeing it waits for the whole device.
constexpr size_t kPinnedBlock = 256;
constexpr size_t kPinnedSlab = 64 * 1024;
std::mutex g_pinned_mu;
std::vector<void*> g_pinned_free;

}  // namespace

void* pinned_take() {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    if (g_pinned_free.empty()) {
        void* slab = nullptr;
        if (cudaHostAlloc(&slab, kPinnedSlab, cudaHostAllocDefault) != cudaSuccess) return nullptr;
        for (size_t off = 0; off < kPinnedSlab; off += kPinnedBlock)
            g_pinned_free.push_back(static_cast<char*>(slab) + off);
    }
    void* p = g_pinned_free.back();
    g_pinned_free.pop_back();
    return p;
}

void pinned_give(void* p) {
    if (p == nullptr) return;
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    g_pinned_free.push_back(p);
}

namespace {

void setup_pool(int device) {
    static std::once_flag once[64];
    if (device < 0 || device >= 64) return;
    std::call_once(once[device], [device]() {
        // Keep freed memory in the stream-ordered pool for this process, so that
        // repeated contexts do not return to the driver for every allocation.
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

// Whether the kernels of the current device may read `p` in place: managed
// memory, or device memory of the current device. Memory of another GPU is
// not (no peer mapping is assumed): it is staged through a copy like host memory.
bool device_accessible(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    if (a.type != cudaMemoryTypeDevice) return false;
    int cur = -1;
    return cudaGetDevice(&cur) == cudaSuccess && a.device == cur;
}

// Device-resident view of a caller array: the array itself if the GPU can
// read it, else a stream-ordered copy that the caller frees after use.
cudaError_t stage(const void* p, size_t bytes, cudaStream_t s, const void** out, std::vector<void*>& temps) {
    if (p == nullptr || bytes == 0 || device_accessible(p)) {
        *out = p;
        return cudaSuccess;
    }
    void* d = nullptr;
    cudaError_t e = cudaMallocAsync(&d, bytes, s);
    if (e) return e;
    temps.push_back(d);
    e = cudaMemcpyAsync(d, p, bytes, cudaMemcpyDefault, s);
    *out = d;
    return e;
}

void free_temps(std::vector<void*>& temps, cudaStream_t s) {
    for (void* p : temps) cudaFreeAsync(p, s);
    temps.clear();
}

void destroy_ctx(bisim_ctx* ctx) {
    if (ctx == nullptr) return;
    dense_release(ctx);
    segment_release(ctx);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(static_cast<cudaStream_t>(ctx->copy_stream));
        cudaStreamDestroy(static_cast<cudaStream_t>(ctx->copy_stream));
    }
    for (void* ev : ctx->copy_events)
        if (ev) cudaEventDestroy(static_cast<cudaEvent_t>(ev));
    // free in the order of the stream the context last worked on, and wait for
    // it: the pool then hands the memory straight to the next context, which a
    // free still pending on the device would make it map afresh
    cudaStream_t s = static_cast<cudaStream_t>(ctx->last_stream);
    for (void* p : ctx->allocs) cudaFreeAsync(p, s);
    if (ctx->dstate) cudaFreeAsync(ctx->dstate, s);
    cudaStreamSynchronize(s);
    pinned_give(ctx->hstate);
    pinned_give(ctx->seg_host);
    delete ctx;
}

bisim_options resolve_options(const bisim_options* in) {
    bisim_options o;
    bisim_default_options(&o);
    if (in != nullptr) o = *in;
    if (o.hash_bits <= 0 || o.hash_bits > 64) o.hash_bits = 64;
    o.small_max_degree = std::min(std::max(o.small_max_degree, 0), 32);
    o.mid_max_degree = std::min(std::max(o.mid_max_degree, 0), kMidMaxN);
    if (o.hub_chunk <= 0) o.hub_chunk = 4096;
    o.hub_chunk = std::min(std::max(o.hub_chunk, 256), kHubChunkMax);
    if (o.k_incremental < 0) o.k_incremental = 0;
    if (o.batch_split < 0) o.batch_split = 0;
    return o;
}

bisim_status new_ctx(bisim_ctx** out, int32_t n, int64_t m, const bisim_options* opt, cudaStream_t s,
                     bisim_ctx** made) {
    if (out == nullptr) return set_error(nullptr, BISIM_EINVAL, "out pointer is NULL");
    *out = nullptr;
    if (n < 0 || m < 0) return set_error(nullptr, BISIM_EINVAL, "negative vertex or edge count");
    if (opt != nullptr && (opt->direction < BISIM_DIR_FORWARD || opt->direction > BISIM_DIR_BOTH))
        return set_error(nullptr, BISIM_EINVAL, "direction must be BISIM_DIR_FORWARD, _BACKWARD or _BOTH");
    if (opt != nullptr && opt->n_label_filter < 0) return set_error(nullptr, BISIM_EINVAL, "n_label_filter < 0");
    bisim_ctx* ctx = new bisim_ctx();
    ctx->last_stream = s;
    ctx->n = n;
    ctx->m = m;
    ctx->opt = resolve_options(opt);
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e) { delete ctx; return cuda_error(nullptr, e, "cudaGetDevice"); }
    setup_pool(ctx->device);
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&ctx->dstate), sizeof(DevState), s))) {
        destroy_ctx(ctx);
        return cuda_error(nullptr, e, "allocate context state");
    }
    ctx->hstate = static_cast<DevState*>(pinned_take());
    if (ctx->hstate == nullptr) {
        destroy_ctx(ctx);
        return set_error(nullptr, BISIM_ENOMEM, "pinned host memory for the context state");
    }
    cudaMemsetAsync(ctx->dstate, 0, sizeof(DevState), s);
    std::memset(ctx->hstate, 0, sizeof(DevState));
    bisim_status st = edge_view_setup(ctx, opt, s);
    if (st != BISIM_OK) {
        const std::string msg = ctx->err;
        destroy_ctx(ctx);
        return set_error(nullptr, st, msg);
    }
    *made = ctx;
    return BISIM_OK;
}

// Builds the context's graph from device COO arrays through its edge view
// (direction and label filter); the view's edge count becomes the context's.
bisim_status build_from_coo_view(bisim_ctx* ctx, const int32_t* src, const int32_t* dst, const int32_t* lab,
                                 cudaStream_t s) {
    if (edge_view_identity(ctx)) return build_from_coo(ctx, src, dst, lab, s);
    EdgeView v;
    bisim_status st = edge_view_coo(ctx, src, dst, lab, ctx->m, nullptr, 0, s, &v);
    if (st == BISIM_OK) {
        ctx->m = v.m;
        st = build_from_coo(ctx, v.src, v.dst, v.lab, s);
    }
    edge_view_free(&v, s);
    return st;
}

bisim_status copy_vertex_arrays(bisim_ctx* ctx, const int32_t* vlabel, const uint8_t* alive, cudaStream_t s) {
    const size_t nv = static_cast<size_t>(std::max(ctx->n, 1));
    cudaError_t e;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->vlabel), sizeof(int32_t) * nv, s))) return cuda_error(ctx, e, "alloc labels");
    if (ctx->n > 0) cudaMemcpyAsync(ctx->vlabel, vlabel, sizeof(int32_t) * ctx->n, cudaMemcpyDefault, s);
    if (alive != nullptr) {
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->alive), nv, s))) return cuda_error(ctx, e, "alloc alive");
        if (ctx->n > 0) cudaMemcpyAsync(ctx->alive, alive, ctx->n, cudaMemcpyDefault, s);
    }
    if ((e = cudaGetLastError())) return cuda_error(ctx, e, "copy vertex arrays");
    return BISIM_OK;
}

// Host graphs of different contexts are copied in one after the other: the
// host link bounds such a copy, and two at once would only share it and
// finish both late, while one after the other lets the first context build
// and refine while the second copies. A context holds the lane from before
// its first copy until the last one has arrived. A wait gives up after a
// minute (the lane then only loses its ordering), so a context that never
// lets go cannot block the others for good.
struct UploadLane {
    std::mutex mu;
    std::condition_variable cv;
    bool busy = false;
};

UploadLane& upload_lane() {
    static UploadLane* lane = new UploadLane();      // never freed: no destructor runs while a thread waits
    return *lane;
}

void lane_take() {
    UploadLane& L = upload_lane();
    std::unique_lock<std::mutex> lk(L.mu);
    L.cv.wait_for(lk, std::chrono::seconds(60), [&] { return !L.busy; });
    L.busy = true;
}

void lane_hand_on() {
    UploadLane& L = upload_lane();
    {
        std::lock_guard<std::mutex> lk(L.mu);
        L.busy = false;
    }
    L.cv.notify_one();
}

struct LaneTurn {
    bool held = false;
    void take() {
        lane_take();
        held = true;
    }
    void give() {
        if (held) lane_hand_on();
        held = false;
    }
    ~LaneTurn() { give(); }
};

// Device buffers for a host COO list (temps[0..2]: sources, targets, labels)
// and their copies on the context's copy stream, each followed by its event
// (copy_events[1..3]); copy_events[0] orders the copies after the buffers'
// allocation on `s`.
bisim_status coo_arrive(bisim_ctx* ctx, const int32_t* src, const int32_t* dst, const int32_t* lab, size_t bytes,
                        cudaStream_t s, std::vector<void*>& temps) {
    cudaError_t e;
    if (ctx->copy_stream == nullptr) {
        if ((e = cudaStreamCreateWithFlags(reinterpret_cast<cudaStream_t*>(&ctx->copy_stream), cudaStreamNonBlocking)))
            return cuda_error(ctx, e, "create copy stream");
        for (void*& ev : ctx->copy_events)
            if ((e = cudaEventCreateWithFlags(reinterpret_cast<cudaEvent_t*>(&ev), cudaEventDisableTiming)))
                return cuda_error(ctx, e, "create copy events");
    }
    cudaStream_t cs = static_cast<cudaStream_t>(ctx->copy_stream);
    const int32_t* host[3] = {src, dst, lab};
    for (int i = 0; i < 3; ++i) {
        void* d = nullptr;
        if ((e = cudaMallocAsync(&d, bytes, s))) return cuda_error(ctx, e, "alloc edge arrays");
        temps.push_back(d);
    }
    cudaEventRecord(static_cast<cudaEvent_t>(ctx->copy_events[0]), s);
    cudaStreamWaitEvent(cs, static_cast<cudaEvent_t>(ctx->copy_events[0]), 0);
    for (int i = 0; i < 3; ++i) {
        if ((e = cudaMemcpyAsync(temps[i], host[i], bytes, cudaMemcpyDefault, cs))) return cuda_error(ctx, e, "copy edge arrays");
        cudaEventRecord(static_cast<cudaEvent_t>(ctx->copy_events[1 + i]), cs);
    }
    return BISIM_OK;
}

bisim_status finish_init(bisim_ctx* ctx, cudaStream_t s) {
    bisim_status st;
    if ((st = alloc_refine_state(ctx, s)) != BISIM_OK) return st;
    if (ctx->opt.mem_budget_bytes > 0 && ctx->device_bytes > ctx->opt.mem_budget_bytes)
        return set_error(ctx, BISIM_ENOMEM, "context exceeds the memory budget");
    if ((st = compute_p0(ctx, s)) != BISIM_OK) return st;
    cudaMemcpyAsync(ctx->P[0], ctx->P0, sizeof(int32_t) * std::max(ctx->n, 1), cudaMemcpyDeviceToDevice, s);
    ctx->cur = 0;
    ctx->stats.n_vertices = ctx->n;
    ctx->stats.n_edges = ctx->m;
    ctx->stats.n_graphs = ctx->n_graphs;
    ctx->stats.device_bytes = ctx->device_bytes;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) return cuda_error(ctx, e, "initialise partition");
    return BISIM_OK;
}

__global__ void k_globalize(const int64_t* __restrict__ voff, const int64_t* __restrict__ eoff, int32_t G,
                            const int32_t* __restrict__ sl, const int32_t* __restrict__ dl, int64_t m,
                            int32_t* __restrict__ src, int32_t* __restrict__ dst, unsigned* err) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int lo = 0, hi = G - 1;   // graph g with eoff[g] <= e < eoff[g+1]
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (eoff[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const int64_t ng = voff[lo + 1] - voff[lo];
        const int32_t a = sl[e], b = dl[e];
        if (a < 0 || a >= ng || b < 0 || b >= ng) {
            atomicOr(err, kErrBadInput);
            src[e] = 0;
            dst[e] = 0;
        } else {
            src[e] = static_cast<int32_t>(voff[lo] + a);
            dst[e] = static_cast<int32_t>(voff[lo] + b);
        }
    }
}

__global__ void k_graph_ids(const int64_t* __restrict__ voff, int32_t G, int32_t n, int32_t* __restrict__ gid) {
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (voff[mid] <= v) lo = mid; else hi = mid - 1;
    }
    gid[v] = lo;
}

}  // namespace

bisim_status set_error(bisim_ctx* ctx, bisim_status st, const std::string& msg) {
    if (ctx != nullptr) ctx->err = msg;
    g_last_error = msg;
    return st;
}

bisim_status cuda_error(bisim_ctx* ctx, cudaError_t e, const char* what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return set_error(ctx, BISIM_ECUDA, msg);
}

cudaError_t ctx_alloc(bisim_ctx* ctx, void** p, size_t bytes, cudaStream_t s) {
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e == cudaSuccess) {
        ctx->allocs.push_back(*p);
        ctx->device_bytes += static_cast<int64_t>(bytes);
    }
    return e;
}

// Rebuilds what depends on the CSR after an update batch changed it: degree
// buckets, signature-list capacity and the label partition.
bisim_status refresh_after_edit(bisim_ctx* ctx, cudaStream_t s) {
    if (!ctx->buckets_dirty) return BISIM_OK;
    cudaError_t e;
    bisim_status st;
    if (ctx->skey != nullptr && ctx->m > ctx->skey_cap) {
        ctx_free(ctx, ctx->skey, sizeof(unsigned long long) * ctx->skey_cap, s);
        ctx->skey = nullptr;
        const int64_t cap = ctx->m + ctx->m / 4 + 1024;
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->skey), sizeof(unsigned long long) * cap, s)))
            return cuda_error(ctx, e, "grow signature lists");
        ctx->skey_cap = cap;
    }
    if ((st = compute_p0(ctx, s)) != BISIM_OK) return st;
    ctx->buckets_dirty = false;
    ctx->stats.device_bytes = ctx->device_bytes;
    return BISIM_OK;
}

// Resets to P_0 and lists the live positions for the dense rounds: all of
// them, or (keep_graph given, batched contexts) only those of the graphs with
// keep_graph[g] != 0; *out_prev is then the block count of P_0 as the rounds
// count it (see dense_keep_graphs).
bisim_status dense_rounds_begin(bisim_ctx* ctx, cudaStream_t s, const uint8_t* keep_graph, int64_t* out_prev,
                                int64_t* out_dropped) {
    bisim_status pst = dense_prepare(ctx, s);
    if (pst != BISIM_OK) return pst;
    if (ctx->opt.mem_budget_bytes > 0 && ctx->device_bytes > ctx->opt.mem_budget_bytes)
        return set_error(ctx, BISIM_ENOMEM, "context exceeds the memory budget");
    if (ctx->n > 0) cudaMemcpyAsync(ctx->P[0], ctx->P0, sizeof(int32_t) * ctx->n, cudaMemcpyDeviceToDevice, s);
    dense_start(ctx, s);
    ctx->cur = 0;
    *out_prev = ctx->last_blocks;   // |P_0|
    *out_dropped = 0;
    if (keep_graph != nullptr) return dense_keep_graphs(ctx, s, keep_graph, out_prev, out_dropped);
    return BISIM_OK;
}

// Refines from the state dense_rounds_begin left: k rounds, or to the fixpoint
// (k = BISIM_FIXPOINT) with at most `cap` rounds. Equal block counts in two
// consecutive rounds prove the fixpoint, since every round refines the
// previous partition.
bisim_status dense_rounds_run(bisim_ctx* ctx, int32_t k, int32_t cap, cudaStream_t s, int64_t prev,
                              int32_t* out_rounds, int32_t* out_executed, int64_t* out_blocks, bool allow_graph) {
    cudaError_t e;
    const bool fixpoint = k == BISIM_FIXPOINT;
    const int32_t limit = fixpoint ? cap : k;
    int32_t rounds = limit, executed = 0;
    bool done = limit <= 0;
    if (!done && allow_graph && dense_graph_usable(ctx)) {
        // the round loop on the device: one graph launch
        GraphRounds g{};
        bisim_status st = dense_graph_rounds(ctx, s, limit, fixpoint, prev, &g);
        if (st != BISIM_OK) return st;
        executed = g.executed;
        if (g.stop == 1) {
            rounds = g.rounds;
            prev = g.blocks;
            done = true;
        } else {
            // the last round met a hash collision (or an error): finish it here
            int64_t blocks = 0;
            if ((st = dense_finish_round(ctx, s, &blocks)) != BISIM_OK) return st;
            if (blocks == prev) {
                rounds = fixpoint ? executed - 1 : k;
                done = true;
            }
            prev = blocks;
        }
    }
    for (int32_t i = executed; !done && i < limit; ++i) {
        int64_t blocks = 0;
        pin_partition_in_l2(ctx, ctx->P[ctx->cur], s);
        bisim_status st = dense_round(ctx, s, &blocks);
        if (st != BISIM_OK) {
            unpin_partition(ctx, s);
            return st;
        }
        ++executed;
        if (blocks == prev) {   // P_{i+1} refines P_i with as many blocks: P_{i+1} = P_i
            rounds = fixpoint ? i : k;
            break;
        }
        prev = blocks;
    }
    unpin_partition(ctx, s);
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "refinement rounds");
    *out_rounds = rounds;
    *out_executed = executed;
    *out_blocks = prev;
    return BISIM_OK;
}

// Resets to P_0 and refines (see dense_rounds_run); batched contexts go to
// segment_rounds.
bisim_status run_rounds(bisim_ctx* ctx, int32_t k, int32_t cap, cudaStream_t s, int32_t* out_rounds,
                        int32_t* out_executed, int64_t* out_blocks, bool allow_graph) {
    if (segment_usable(ctx)) return segment_rounds(ctx, k, cap, s, out_rounds, out_executed, out_blocks);
    int64_t prev = 0, dropped = 0;
    bisim_status st = dense_rounds_begin(ctx, s, nullptr, &prev, &dropped);
    if (st != BISIM_OK) return st;
    int32_t rounds = 0, executed = 0;
    if ((st = dense_rounds_run(ctx, k, cap, s, prev, &rounds, &executed, &prev, allow_graph)) != BISIM_OK) return st;
    ctx->cur_k = rounds;
    ctx->stats.rounds = rounds;
    ctx->stats.rounds_executed = executed;
    ctx->stats.num_blocks = prev;
    *out_rounds = rounds;
    *out_executed = executed;
    *out_blocks = prev;
    return BISIM_OK;
}

}  // namespace bisim

using namespace bisim;

extern "C" {

bisim_status bisim_retune(bisim_ctx* ctx, const bisim_options* opt, void* stream) {
    if (ctx == nullptr) return set_error(nullptr, BISIM_EINVAL, "ctx is NULL");
    if (opt == nullptr) return set_error(ctx, BISIM_EINVAL, "opt is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ctx->last_stream = stream;
    bisim_status st;
    // the new layout is built from the vertex-ordered CSR: make it from the
    // current layout while that one is still valid
    if ((st = refresh_after_edit(ctx, s)) != BISIM_OK || (st = dense_prepare(ctx, s)) != BISIM_OK ||
        (st = ensure_vertex_csr(ctx, s)) != BISIM_OK)
        return st;
    cudaError_t e;
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "retune");
    const bisim_options o = resolve_options(opt);
    ctx->opt.small_max_degree = o.small_max_degree;
    ctx->opt.mid_max_degree = o.mid_max_degree;
    ctx->opt.hub_chunk = o.hub_chunk;
    ctx->opt.batch_split = o.batch_split;
    ctx->dense_ready = false;        // the next run rebuilds the layout with them
    return BISIM_OK;
}

void bisim_default_options(bisim_options* opt) {
    if (opt == nullptr) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->k_incremental = 2;
    opt->hash_bits = 64;
    opt->small_max_degree = 32;
    opt->mid_max_degree = kMidMaxN;
    opt->hub_chunk = 4096;
    opt->mem_budget_bytes = 0;
    opt->batch_split = 0;
}

bisim_status summarize_init(bisim_ctx** out, int32_t n_vertices, int64_t n_edges, const int64_t* row_ptr,
                            const int32_t* col, const int32_t* edge_label, const int32_t* vertex_label,
                            const uint8_t* alive, const bisim_options* opt, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bisim_ctx* ctx = nullptr;
    bisim_status st = new_ctx(out, n_vertices, n_edges, opt, s, &ctx);
    if (st != BISIM_OK) return st;
    if (row_ptr == nullptr || (n_vertices > 0 && vertex_label == nullptr) ||
        (n_edges > 0 && (col == nullptr || edge_label == nullptr))) {
        destroy_ctx(ctx);
        return set_error(nullptr, BISIM_EINVAL, "a required array is NULL");
    }
    if (!edge_view_identity(ctx) && (st = copy_vertex_arrays(ctx, vertex_label, alive, s)) == BISIM_OK) {
        // another direction or a label filter: the CSR's edges as a list, then the view's COO path
        std::vector<void*> temps;
        const void *drp = nullptr, *dc = nullptr, *dl = nullptr;
        int32_t* dsrc = nullptr;
        cudaError_t e;
        const size_t eb = sizeof(int32_t) * static_cast<size_t>(n_edges);
        if ((e = stage(row_ptr, sizeof(int64_t) * (static_cast<size_t>(n_vertices) + 1), s, &drp, temps)) ||
            (e = stage(col, eb, s, &dc, temps)) || (e = stage(edge_label, eb, s, &dl, temps)) ||
            (e = cudaMallocAsync(reinterpret_cast<void**>(&dsrc), std::max<size_t>(eb, 4), s)))
            st = cuda_error(ctx, e, "stage CSR arrays");
        if (st == BISIM_OK)
            st = csr_sources(ctx, static_cast<const int64_t*>(drp), n_vertices, n_edges, dsrc, s);
        if (st == BISIM_OK)
            st = build_from_coo_view(ctx, dsrc, static_cast<const int32_t*>(dc), static_cast<const int32_t*>(dl), s);
        if (dsrc) cudaFreeAsync(dsrc, s);
        free_temps(temps, s);
        if (st == BISIM_OK && (st = finish_init(ctx, s)) == BISIM_OK) {
            *out = ctx;
            return BISIM_OK;
        }
    } else if (edge_view_identity(ctx) && (st = copy_vertex_arrays(ctx, vertex_label, alive, s)) == BISIM_OK &&
               (st = build_from_csr(ctx, row_ptr, col, edge_label, s)) == BISIM_OK &&
               (st = finish_init(ctx, s)) == BISIM_OK) {
        *out = ctx;
        return BISIM_OK;
    }
    std::string msg = ctx->err;
    destroy_ctx(ctx);
    return set_error(nullptr, st, msg);
}

bisim_status summarize_init_coo(bisim_ctx** out, int32_t n_vertices, int64_t n_edges, const int32_t* src,
                                const int32_t* dst, const int32_t* edge_label, const int32_t* vertex_label,
                                const uint8_t* alive, const bisim_options* opt, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bisim_ctx* ctx = nullptr;
    bisim_status st = new_ctx(out, n_vertices, n_edges, opt, s, &ctx);
    if (st != BISIM_OK) return st;
    if ((n_vertices > 0 && vertex_label == nullptr) ||
        (n_edges > 0 && (src == nullptr || dst == nullptr || edge_label == nullptr))) {
        destroy_ctx(ctx);
        return set_error(nullptr, BISIM_EINVAL, "a required array is NULL");
    }
    std::vector<void*> temps;
    const void *ds = nullptr, *dd = nullptr, *dl = nullptr;
    cudaError_t e;
    const size_t eb = sizeof(int32_t) * static_cast<size_t>(n_edges);
    if (n_edges > 0 && edge_view_identity(ctx) && !device_accessible(src) && !device_accessible(dst) &&
        !device_accessible(edge_label)) {
        // a host list: copied in on a stream of its own, sources first, while
        // P_0 and then the sources' part of the build run on `stream`; the
        // upload lane is held until the last array has arrived
        LaneTurn turn;
        turn.take();
        if ((st = copy_vertex_arrays(ctx, vertex_label, alive, s)) == BISIM_OK) st = coo_arrive(ctx, src, dst, edge_label, eb, s, temps);
        if (st == BISIM_OK) st = finish_init(ctx, s);
        if (st == BISIM_OK) {
            CooArrival arr;
            arr.src = static_cast<cudaEvent_t>(ctx->copy_events[1]);
            arr.dst = static_cast<cudaEvent_t>(ctx->copy_events[2]);
            arr.lab = static_cast<cudaEvent_t>(ctx->copy_events[3]);
            arr.arrived = [](void* t) { static_cast<LaneTurn*>(t)->give(); };
            arr.arrived_arg = &turn;
            st = build_from_coo(ctx, static_cast<const int32_t*>(temps[0]), static_cast<const int32_t*>(temps[1]),
                                static_cast<const int32_t*>(temps[2]), s, &arr);
        }
        turn.give();
        // no copy may still write a buffer that is freed (a failed build can
        // return before it waited for the last of them)
        if (st != BISIM_OK && ctx->copy_stream) cudaStreamSynchronize(static_cast<cudaStream_t>(ctx->copy_stream));
        free_temps(temps, s);
        if (st == BISIM_OK) {
            ctx->stats.device_bytes = ctx->device_bytes;
            if ((e = cudaStreamSynchronize(s))) st = cuda_error(ctx, e, "build from a host list");
        }
        if (st == BISIM_OK) {
            *out = ctx;
            return BISIM_OK;
        }
        std::string msg = ctx->err;
        destroy_ctx(ctx);
        return set_error(nullptr, st, msg);
    }
    if ((st = copy_vertex_arrays(ctx, vertex_label, alive, s)) == BISIM_OK) {
        if ((e = stage(src, eb, s, &ds, temps)) || (e = stage(dst, eb, s, &dd, temps)) ||
            (e = stage(edge_label, eb, s, &dl, temps)))
            st = cuda_error(ctx, e, "stage edge arrays");
    }
    if (st == BISIM_OK)
        st = build_from_coo_view(ctx, static_cast<const int32_t*>(ds), static_cast<const int32_t*>(dd),
                                 static_cast<const int32_t*>(dl), s);
    free_temps(temps, s);
    if (st == BISIM_OK && (st = finish_init(ctx, s)) == BISIM_OK) {
        *out = ctx;
        return BISIM_OK;
    }
    std::string msg = ctx->err;
    destroy_ctx(ctx);
    return set_error(nullptr, st, msg);
}

bisim_status summarize_init_batched(bisim_ctx** out, int32_t n_graphs, const int64_t* vertex_offsets,
                                    const int64_t* edge_offsets, const int32_t* src_local,
                                    const int32_t* dst_local, const int32_t* edge_label,
                                    const int32_t* vertex_label, const bisim_options* opt, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (out == nullptr) return set_error(nullptr, BISIM_EINVAL, "out pointer is NULL");
    *out = nullptr;
    if (n_graphs <= 0 || vertex_offsets == nullptr || edge_offsets == nullptr)
        return set_error(nullptr, BISIM_EINVAL, "batched init needs n_graphs >= 1 and both offset arrays");
    std::vector<int64_t> hv(n_graphs + 1), he(n_graphs + 1);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(hv.data(), vertex_offsets, sizeof(int64_t) * (n_graphs + 1), cudaMemcpyDefault, s)) ||
        (e = cudaMemcpyAsync(he.data(), edge_offsets, sizeof(int64_t) * (n_graphs + 1), cudaMemcpyDefault, s)) ||
        (e = cudaStreamSynchronize(s)))
        return cuda_error(nullptr, e, "read batch offsets");
    if (hv[0] != 0 || he[0] != 0) return set_error(nullptr, BISIM_EINVAL, "offsets must start at 0");
    for (int32_t g = 0; g < n_graphs; ++g)
        if (hv[g + 1] < hv[g] || he[g + 1] < he[g]) return set_error(nullptr, BISIM_EINVAL, "offsets must be non-decreasing");
    if (hv[n_graphs] > INT32_MAX) return set_error(nullptr, BISIM_EINVAL, "more than 2^31-1 vertices in total");
    const int32_t n = static_cast<int32_t>(hv[n_graphs]);
    const int64_t m = he[n_graphs];
    bisim_ctx* ctx = nullptr;
    bisim_status st = new_ctx(out, n, m, opt, s, &ctx);
    if (st != BISIM_OK) return st;
    ctx->n_graphs = n_graphs;
    if ((n > 0 && vertex_label == nullptr) || (m > 0 && (src_local == nullptr || dst_local == nullptr || edge_label == nullptr))) {
        destroy_ctx(ctx);
        return set_error(nullptr, BISIM_EINVAL, "a required array is NULL");
    }
    std::vector<void*> temps;
    const void *ds = nullptr, *dd = nullptr, *dl = nullptr;
    const size_t eb = sizeof(int32_t) * static_cast<size_t>(m);
    int32_t* gsrc = nullptr;
    int32_t* gdst = nullptr;
    int64_t* deoff = nullptr;
    if ((st = copy_vertex_arrays(ctx, vertex_label, nullptr, s)) == BISIM_OK) {
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->voff), sizeof(int64_t) * (n_graphs + 1), s)) ||
            (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->gid), sizeof(int32_t) * std::max(n, 1), s)) ||
            (e = cudaMallocAsync(reinterpret_cast<void**>(&deoff), sizeof(int64_t) * (n_graphs + 1), s)) ||
            (e = cudaMallocAsync(reinterpret_cast<void**>(&gsrc), std::max<size_t>(eb, 4), s)) ||
            (e = cudaMallocAsync(reinterpret_cast<void**>(&gdst), std::max<size_t>(eb, 4), s)) ||
            (e = stage(src_local, eb, s, &ds, temps)) || (e = stage(dst_local, eb, s, &dd, temps)) ||
            (e = stage(edge_label, eb, s, &dl, temps)))
            st = cuda_error(ctx, e, "stage batched arrays");
    }
    if (st == BISIM_OK) {
        cudaMemcpyAsync(ctx->voff, hv.data(), sizeof(int64_t) * (n_graphs + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(deoff, he.data(), sizeof(int64_t) * (n_graphs + 1), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(&ctx->dstate->error, 0, sizeof(unsigned), s);
        BISIM_SITE(site_g, "batch_graph_ids");
        BISIM_SITE(site_e, "batch_globalize");
        if (n > 0)
            Launch(site_g, s, n, 0, 4.0 * n),
            k_graph_ids<<<(n + 255) / 256, 256, 0, s>>>(ctx->voff, n_graphs, n, ctx->gid);
        if (m > 0)
            Launch(site_e, s, 0, m, 16.0 * m),
            k_globalize<<<static_cast<unsigned>(std::min<int64_t>((m + 255) / 256, 1 << 16)), 256, 0, s>>>(
                ctx->voff, deoff, n_graphs, static_cast<const int32_t*>(ds), static_cast<const int32_t*>(dd), m,
                gsrc, gdst, &ctx->dstate->error);
        cudaMemcpyAsync(ctx->hstate, ctx->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s))) st = cuda_error(ctx, e, "globalize batched edges");
        else if (ctx->hstate->error & kErrBadInput) st = set_error(ctx, BISIM_EINVAL, "a graph-local edge endpoint is out of range");
    }
    EdgeView view;
    const int32_t* bl = static_cast<const int32_t*>(dl);
    if (st == BISIM_OK && !edge_view_identity(ctx)) {
        // another direction or a label filter: the view keeps every graph's edges together
        if ((st = edge_view_coo(ctx, gsrc, gdst, bl, m, deoff, n_graphs, s, &view)) == BISIM_OK) {
            ctx->m = view.m;
            if ((e = cudaMemcpyAsync(he.data(), view.eoff, sizeof(int64_t) * (n_graphs + 1), cudaMemcpyDeviceToHost, s)) ||
                (e = cudaStreamSynchronize(s)))
                st = cuda_error(ctx, e, "read view offsets");
        }
    }
    if (st == BISIM_OK)
        st = build_from_coo(ctx, view.src ? view.src : gsrc, view.src ? view.dst : gdst, view.src ? view.lab : bl, s);
    edge_view_free(&view, s);
    if (st == BISIM_OK) st = dense_region_table(ctx, hv.data(), n_graphs, s);
    if (st == BISIM_OK) st = segment_init(ctx, hv.data(), he.data(), n_graphs, s);
    free_temps(temps, s);
    if (deoff) cudaFreeAsync(deoff, s);
    if (gsrc) cudaFreeAsync(gsrc, s);
    if (gdst) cudaFreeAsync(gdst, s);
    if (st == BISIM_OK && (st = finish_init(ctx, s)) == BISIM_OK) {
        *out = ctx;
        return BISIM_OK;
    }
    std::string msg = ctx->err;
    destroy_ctx(ctx);
    return set_error(nullptr, st, msg);
}

bisim_status bisim_iterate(bisim_ctx* ctx, int32_t k, int32_t cap, int32_t* out_rounds, int64_t* out_num_blocks,
                           void* stream) {
    if (ctx == nullptr) return set_error(nullptr, BISIM_EINVAL, "ctx is NULL");
    ctx->last_stream = stream;
    if (k < BISIM_FIXPOINT) return set_error(ctx, BISIM_EINVAL, "k must be >= 0 or BISIM_FIXPOINT");
    if (k == BISIM_FIXPOINT && cap < 0) return set_error(ctx, BISIM_EINVAL, "cap must be >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bisim_status st;
    if ((st = refresh_after_edit(ctx, s)) != BISIM_OK) return st;
    int32_t rounds = 0, executed = 0;
    int64_t blocks = 0;
    if ((st = run_rounds(ctx, k, cap, s, &rounds, &executed, &blocks)) != BISIM_OK) return st;
    if (out_rounds) *out_rounds = rounds;
    if (out_num_blocks) *out_num_blocks = blocks;
    return BISIM_OK;
}

bisim_status apply_updates(bisim_ctx* ctx, const bisim_op* ops, int64_t n_ops, void* stream) {
    if (ctx == nullptr) return set_error(nullptr, BISIM_EINVAL, "ctx is NULL");
    ctx->last_stream = stream;
    if (n_ops < 0 || (n_ops > 0 && ops == nullptr)) return set_error(ctx, BISIM_EINVAL, "invalid op array");
    if (ctx->gid != nullptr) return set_error(ctx, BISIM_ESTATE, "apply_updates is not supported on batched contexts");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    bisim_status st;
    const bool full = (ctx->opt.flags & BISIM_FLAG_FULL_RECOMPUTE) != 0;
    // batches edit the incremental path's row store in place once its state is
    // built; otherwise (and for full recomputes) they rewrite the CSR
    const bool incremental = !full && ctx->inc_k == ctx->opt.k_incremental && ctx->store_ready;
    if (!incremental && (st = ensure_vertex_csr(ctx, s)) != BISIM_OK) return st;
    std::vector<void*> temps;
    const void* d_ops = nullptr;
    if (n_ops > 0) {
        if ((e = stage(ops, sizeof(bisim_op) * static_cast<size_t>(n_ops), s, &d_ops, temps)))
            return cuda_error(ctx, e, "stage update batch");
        if (!edge_view_identity(ctx)) {
            // another direction or a label filter: the operations on the context's own edge list
            bisim_op* vops = nullptr;
            int64_t vn = 0;
            st = edge_view_ops(ctx, static_cast<const bisim_op*>(d_ops), n_ops, s, &vops, &vn);
            if (vops) temps.push_back(vops);
            if (st != BISIM_OK) {
                free_temps(temps, s);
                return st;
            }
            d_ops = vops;
            n_ops = vn;
        }
    }
    if (n_ops == 0) free_temps(temps, s);
    if (n_ops > 0) {
        uint8_t* flags = nullptr;
        // three flag arrays of n + 1 bytes, each starting on a 256-byte boundary
        // (the frontier kernels read them 16 bytes at a time)
        const size_t fs = (static_cast<size_t>(ctx->n + 1) + 255) & ~size_t(255);
        const size_t fb = 3 * fs;
        if ((e = cudaMallocAsync(reinterpret_cast<void**>(&flags), fb, s))) {
            free_temps(temps, s);
            return cuda_error(ctx, e, "alloc update flags");
        }
        cudaMemsetAsync(flags, 0, fb, s);
        uint8_t* vchanged = flags;
        uint8_t* rowchg = flags + fs;
        uint8_t* killed = flags + 2 * fs;
        const bisim_op* dops = static_cast<const bisim_op*>(d_ops);
        st = incremental ? apply_ops_to_store(ctx, dops, n_ops, vchanged, rowchg, killed, s)
                         : apply_ops_to_graph(ctx, dops, n_ops, vchanged, rowchg, killed, s);
        free_temps(temps, s);
        if (st == BISIM_OK) {
            ctx->buckets_dirty = true;
            ctx->dense_ready = false;
            if (incremental) {
                st = inc_update(ctx, vchanged, rowchg, n_ops, s);
            } else {
                // the CSR moved on: the row store and any incremental state describe the old graph
                inc_release(ctx, s);
                store_release(ctx, s);
            }
        }
        cudaFreeAsync(flags, s);
        if (st != BISIM_OK) return st;
        if (incremental) return BISIM_OK;
    }
    if (!full) {
        // first batch (or k changed): build the incremental state of the current graph
        if (ctx->inc_k != ctx->opt.k_incremental || !ctx->store_ready) return inc_build(ctx, s);
        return write_current(ctx, s);
    }
    // full recompute at k_incremental rounds
    if ((st = refresh_after_edit(ctx, s)) != BISIM_OK) return st;
    int32_t rounds = 0, executed = 0;
    int64_t blocks = 0;
    if ((st = run_rounds(ctx, ctx->opt.k_incremental, 0, s, &rounds, &executed, &blocks, false)) != BISIM_OK)
        return st;
    ctx->stats.last_frontier = ctx->n;
    return BISIM_OK;
}

// ----------------------------------------------------------------------------- state export / import

namespace {

// Fixed part of an exported state; the arrays follow it, each starting on an
// 8-byte boundary, in the order of state_arrays().
struct StateHeader {
    char magic[8];                 // "BISIMST1"
    uint32_t version;              // 1
    uint32_t header_bytes;
    int32_t n;
    int32_t inc_k;                 // levels of incremental state, -1: none
    int64_t m;                     // edges of the context's own edge list (after direction and filter)
    int32_t k_incremental, hash_bits, small_max_degree, mid_max_degree, hub_chunk, flags, direction, nfilter;
    int64_t mem_budget_bytes;
    int64_t bcap;
    uint64_t isize;
    int64_t bnext[kMaxIncLevels + 1];
    int64_t itomb[kMaxIncLevels + 1];
    int32_t cur_k;
    int32_t has_alive;
    int64_t updates_applied;
    int64_t num_blocks;
    int32_t rounds, rounds_executed;
};

constexpr char kStateMagic[8] = {'B', 'I', 'S', 'I', 'M', 'S', 'T', '1'};

struct StateArray {
    void* dev;                     // device source (export) or destination (import); null: host-side item
    size_t bytes;
};

size_t pad8(size_t b) { return (b + 7) & ~size_t(7); }

// The arrays of a state in blob order: filter, vertex labels, alive flags,
// current partition, CSR (row_ptr, col, labels), then per level block ids,
// |S|, stale flags, block records (key, count, smallest member) and index
// (key, block).
std::vector<StateArray> state_arrays(const bisim_ctx* ctx, const StateHeader& h) {
    const size_t n = static_cast<size_t>(h.n), m = static_cast<size_t>(h.m);
    std::vector<StateArray> a;
    a.push_back({ctx->dfilter, 4 * static_cast<size_t>(h.nfilter)});
    a.push_back({ctx->vlabel, 4 * n});
    a.push_back({ctx->alive, h.has_alive ? n : 0});
    a.push_back({ctx->P[ctx->cur], 4 * n});
    a.push_back({ctx->row_ptr, 8 * (n + 1)});
    a.push_back({ctx->col, 4 * m});
    a.push_back({ctx->elab, 4 * m});
    for (int j = 0; j <= h.inc_k; ++j) {
        a.push_back({ctx->lid[j], 4 * n});
        a.push_back({ctx->lcnt[j], 4 * n});
        a.push_back({ctx->lstale[j], n});
        a.push_back({ctx->bkey[j], 8 * static_cast<size_t>(h.bcap)});
        a.push_back({ctx->bcnt[j], 4 * static_cast<size_t>(h.bcap)});
        a.push_back({ctx->bmin[j], 4 * static_cast<size_t>(h.bcap)});
        a.push_back({ctx->ikey[j], 8 * h.isize});
        a.push_back({ctx->ibid[j], 4 * h.isize});
    }
    return a;
}

size_t state_bytes(const std::vector<StateArray>& a) {
    size_t b = pad8(sizeof(StateHeader));
    for (const auto& x : a) b += pad8(x.bytes);
    return b;
}

}  // namespace

bisim_status bisim_export_state(bisim_ctx* ctx, void* buf, int64_t capacity, int64_t* out_bytes, void* stream) {
    if (ctx == nullptr) return set_error(nullptr, BISIM_EINVAL, "ctx is NULL");
    ctx->last_stream = stream;
    if (out_bytes == nullptr || capacity < 0) return set_error(ctx, BISIM_EINVAL, "invalid size arguments");
    if (ctx->gid != nullptr) return set_error(ctx, BISIM_ESTATE, "batched contexts have no exportable state");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bisim_status st;
    // the CSR of the current graph (rebuilt from the row store when batches edited it)
    if ((st = refresh_after_edit(ctx, s)) != BISIM_OK || (st = ensure_vertex_csr(ctx, s)) != BISIM_OK) return st;
    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kStateMagic, 8);
    h.version = 1;
    h.header_bytes = sizeof(StateHeader);
    h.n = ctx->n;
    h.m = ctx->m;
    h.inc_k = ctx->inc_k == ctx->opt.k_incremental && ctx->store_ready ? ctx->inc_k : -1;
    h.k_incremental = ctx->opt.k_incremental;
    h.hash_bits = ctx->opt.hash_bits;
    h.small_max_degree = ctx->opt.small_max_degree;
    h.mid_max_degree = ctx->opt.mid_max_degree;
    h.hub_chunk = ctx->opt.hub_chunk;
    h.flags = ctx->opt.flags;
    h.direction = ctx->opt.direction;
    h.nfilter = ctx->nfilter;
    h.mem_budget_bytes = ctx->opt.mem_budget_bytes;
    h.bcap = h.inc_k >= 0 ? ctx->bcap : 0;
    h.isize = h.inc_k >= 0 ? ctx->isize : 0;
    for (int j = 0; j <= kMaxIncLevels; ++j) {
        h.bnext[j] = ctx->bnext[j];
        h.itomb[j] = ctx->itomb[j];
    }
    h.cur_k = ctx->cur_k;
    h.has_alive = ctx->alive != nullptr ? 1 : 0;
    h.updates_applied = ctx->stats.updates_applied;
    h.num_blocks = ctx->stats.num_blocks;
    h.rounds = ctx->stats.rounds;
    h.rounds_executed = ctx->stats.rounds_executed;
    const std::vector<StateArray> arrays = state_arrays(ctx, h);
    const size_t total = state_bytes(arrays);
    *out_bytes = static_cast<int64_t>(total);
    if (buf == nullptr || capacity < static_cast<int64_t>(total)) return BISIM_OK;
    char* p = static_cast<char*>(buf);
    std::memset(p, 0, pad8(sizeof(StateHeader)));
    std::memcpy(p, &h, sizeof(h));
    size_t off = pad8(sizeof(StateHeader));
    cudaError_t e;
    for (const auto& x : arrays) {
        if (x.bytes > 0 && (e = cudaMemcpyAsync(p + off, x.dev, x.bytes, cudaMemcpyDefault, s)))
            return cuda_error(ctx, e, "export state");
        off += pad8(x.bytes);
    }
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "export state");
    return BISIM_OK;
}

bisim_status bisim_import_state(bisim_ctx** out, const void* buf, int64_t bytes, void* stream) {
    if (out == nullptr) return set_error(nullptr, BISIM_EINVAL, "out pointer is NULL");
    *out = nullptr;
    if (buf == nullptr || bytes < static_cast<int64_t>(sizeof(StateHeader)))
        return set_error(nullptr, BISIM_EINVAL, "state buffer too small");
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.version != 1 || h.header_bytes != sizeof(StateHeader))
        return set_error(nullptr, BISIM_EINVAL, "not an exported bisim state (magic or version)");
    if (h.n < 0 || h.m < 0 || h.inc_k < -1 || h.inc_k > kMaxIncLevels || h.nfilter < 0 || h.bcap < 0 ||
        (h.inc_k >= 0 && (h.bcap < 2 * static_cast<int64_t>(h.n) || h.isize == 0 || (h.isize & (h.isize - 1)))))
        return set_error(nullptr, BISIM_EINVAL, "exported state header is inconsistent");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // sizes from the header alone, before anything is allocated
    bisim_ctx probe;
    probe.n = h.n;
    const std::vector<StateArray> sizes = state_arrays(&probe, h);
    if (static_cast<int64_t>(state_bytes(sizes)) != bytes)
        return set_error(nullptr, BISIM_EINVAL, "exported state has the wrong length");
    const char* p = static_cast<const char*>(buf);
    std::vector<const char*> at;
    size_t off = pad8(sizeof(StateHeader));
    for (const auto& x : sizes) {
        at.push_back(p + off);
        off += pad8(x.bytes);
    }
    bisim_options o;
    bisim_default_options(&o);
    o.k_incremental = h.k_incremental;
    o.hash_bits = h.hash_bits;
    o.small_max_degree = h.small_max_degree;
    o.mid_max_degree = h.mid_max_degree;
    o.hub_chunk = h.hub_chunk;
    o.flags = h.flags;
    o.direction = h.direction;
    o.n_label_filter = h.nfilter;
    o.label_filter = reinterpret_cast<const int32_t*>(at[0]);
    o.mem_budget_bytes = h.mem_budget_bytes;
    bisim_ctx* ctx = nullptr;
    bisim_status st = new_ctx(out, h.n, h.m, &o, s, &ctx);
    if (st != BISIM_OK) return st;
    // the exported edge list already has the direction and filter applied: built as given
    const uint8_t* alive = h.has_alive ? reinterpret_cast<const uint8_t*>(at[2]) : nullptr;
    if ((st = copy_vertex_arrays(ctx, reinterpret_cast<const int32_t*>(at[1]), alive, s)) == BISIM_OK &&
        (st = build_from_csr(ctx, reinterpret_cast<const int64_t*>(at[4]), reinterpret_cast<const int32_t*>(at[5]),
                             reinterpret_cast<const int32_t*>(at[6]), s)) == BISIM_OK &&
        (st = finish_init(ctx, s)) == BISIM_OK && h.inc_k >= 0)
        st = inc_alloc_levels(ctx, h.inc_k, h.bcap, h.isize, s);
    cudaError_t e = cudaSuccess;
    if (st == BISIM_OK) {
        const std::vector<StateArray> dst = state_arrays(ctx, h);
        for (size_t i = 7; i < dst.size() && !e; ++i)       // the levels
            if (dst[i].bytes > 0) e = cudaMemcpyAsync(dst[i].dev, at[i], dst[i].bytes, cudaMemcpyHostToDevice, s);
        if (!e && h.n > 0) e = cudaMemcpyAsync(ctx->P[ctx->cur], at[3], 4 * static_cast<size_t>(h.n), cudaMemcpyHostToDevice, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) st = cuda_error(ctx, e, "import state");
    }
    if (st != BISIM_OK) {
        const std::string msg = ctx->err;
        destroy_ctx(ctx);
        return set_error(nullptr, st, msg);
    }
    for (int j = 0; j <= kMaxIncLevels; ++j) ctx->itomb[j] = h.itomb[j];
    if (h.inc_k >= 0 && (st = inc_set_next_ids(ctx, h.bnext, s)) != BISIM_OK) {
        const std::string msg = ctx->err;
        destroy_ctx(ctx);
        return set_error(nullptr, st, msg);
    }
    ctx->cur_k = h.cur_k;
    ctx->stats.updates_applied = h.updates_applied;
    ctx->stats.num_blocks = h.num_blocks;
    ctx->stats.rounds = h.rounds;
    ctx->stats.rounds_executed = h.rounds_executed;
    *out = ctx;
    return BISIM_OK;
}

bisim_status get_partition(bisim_ctx* ctx, int32_t* block, void* stream) {
    if (ctx == nullptr) return set_error(nullptr, BISIM_EINVAL, "ctx is NULL");
    ctx->last_stream = stream;
    if (block == nullptr && ctx->n > 0) return set_error(ctx, BISIM_EINVAL, "output is NULL");
    if (ctx->n == 0) return BISIM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const int32_t* src = ctx->P[ctx->cur];
    if (ctx->gid != nullptr) {
        int32_t* tmp = ctx->P[ctx->cur ^ 1];   // scratch: the other partition buffer
        launch_local_ids(ctx, tmp, s);
        src = tmp;
    }
    if ((e = cudaMemcpyAsync(block, src, sizeof(int32_t) * ctx->n, cudaMemcpyDefault, s)))
        return cuda_error(ctx, e, "copy partition");
    if (ctx->gid != nullptr) {
        // the scratch buffer is the next round's output; make sure the copy is done first
        if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "copy partition");
    }
    return BISIM_OK;
}

bisim_status bisim_get_stats(const bisim_ctx* ctx, bisim_stats* out) {
    if (ctx == nullptr || out == nullptr) return set_error(nullptr, BISIM_EINVAL, "NULL argument");
    *out = ctx->stats;
    out->device_bytes = ctx->device_bytes;         // what the context holds now
    return BISIM_OK;
}

bisim_status summarize_destroy(bisim_ctx* ctx) {
    destroy_ctx(ctx);
    return BISIM_OK;
}

const char* bisim_last_error(const bisim_ctx* ctx) {
    if (ctx != nullptr) return ctx->err.empty() ? "no error" : ctx->err.c_str();
    return g_last_error.c_str();
}

}  // extern "C"
