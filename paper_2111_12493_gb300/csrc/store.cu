// The incremental path's dynamic adjacency (Section 3.2: the graph evolves by
// batches of additions and deletions, and only the vertices near a change are
// revisited).
//
// Every vertex has an out-row of packed (label << 32 | target) entries and an
// in-row of source vertices, each with spare capacity, in two pools. A batch
// deletes out-entries in place (they become kRowTomb), appends added edges to
// both rows, and moves a row that runs out of room to the pool's tail
// (compacting it on the way); so a batch costs time in proportion to the rows
// it touches, not to the size of the graph. In-rows are append-only: the
// in-entry of a deleted edge stays, so an in-row names a superset of the
// current in-neighbours, which is all the frontier search needs. Edges into a
// dead vertex stay in their source rows too and are skipped by every reader
// (the dead vertex has no block id); they are purged when the vertex is added
// again.
//
// The CSR (row_ptr / col / elab) stays the input of the full-recompute paths;
// after batches edited the store it is rebuilt from it on first use.
#include <algorithm>

#include "common.cuh"
#include "prof.cuh"
#include "rows.cuh"

namespace bisim {

namespace {

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
unsigned grid_for(int64_t n, int threads) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(cdiv(n, threads), 1 << 20)));
}

__device__ __forceinline__ unsigned lane_of() { return threadIdx.x & 31u; }

// Capacity of a row holding d entries: a quarter more, at least two spare.
__host__ __device__ __forceinline__ int32_t row_capacity(int64_t d) {
    return static_cast<int32_t>(d + d / 4 + 2);
}

__global__ void k_store_out_caps(const int64_t* __restrict__ rp, int32_t n, int32_t* __restrict__ xlen,
                                 int32_t* __restrict__ xcap, int64_t* __restrict__ caps) {
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v > n) return;
    if (v == n) {
        caps[v] = 0;
        return;
    }
    const int64_t d = rp[v + 1] - rp[v];
    xlen[v] = static_cast<int32_t>(d);
    xcap[v] = row_capacity(d);
    caps[v] = xcap[v];
}

// In-degrees, one atomic per run of equal targets in a warp (popular targets
// receive millions of edges).
__global__ void k_store_in_degrees(const int32_t* __restrict__ col, int64_t m, int32_t* __restrict__ indeg) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; e0 < m; e0 += stride) {
        const int64_t e = e0 + threadIdx.x;
        const int32_t w = e < m ? col[e] : -1 - static_cast<int32_t>(lane_of());
        const unsigned peers = __match_any_sync(0xffffffffu, w);
        if (e < m && static_cast<int>(lane_of()) == __ffs(peers) - 1) atomicAdd(&indeg[w], __popc(peers));
    }
}

__global__ void k_store_in_caps(int32_t n, int32_t* __restrict__ ylen, int32_t* __restrict__ ycap,
                                int64_t* __restrict__ caps) {
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v > n) return;
    if (v == n) {
        caps[v] = 0;
        return;
    }
    ycap[v] = row_capacity(ylen[v]);
    caps[v] = ycap[v];
    ylen[v] = 0;                     // refilled by k_store_fill
}

// Copies every CSR edge into its out-row (same order) and its target's in-row.
__global__ void k_store_fill(const int64_t* __restrict__ rp, const int32_t* __restrict__ esrc,
                             const int32_t* __restrict__ col, const int32_t* __restrict__ elab, int64_t m,
                             StoreView S) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const unsigned lane = lane_of();
    for (int64_t e0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; e0 < m; e0 += stride) {
        const int64_t e = e0 + threadIdx.x;
        int32_t u = 0, w = -1 - static_cast<int32_t>(lane);
        if (e < m) {
            u = esrc[e];
            w = col[e];
            S.xpe[S.xro[u] + (e - rp[u])] = pack_edge(elab[e], w);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, w);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (e < m && static_cast<int>(lane) == leader) base = atomicAdd(&S.ylen[w], __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (e < m) S.ype[S.yro[w] + base + __popc(peers & ((1u << lane) - 1u))] = u;
    }
}

// ----------------------------------------------------------------------------- CSR from the store

__global__ void k_store_row_tasks(int32_t n, const uint8_t* __restrict__ alive, StoreView S, TierLists L) {
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool has = v < n && (alive == nullptr || alive[v]);
    RowTask t{0, 0, static_cast<int32_t>(v)};
    if (has) {
        t.off = S.xro[v];
        t.len = S.xlen[v];
    }
    tier_push(L, has, t);
}

// An out-entry counts when it was not deleted and its target is live.
__device__ __forceinline__ bool entry_live(unsigned long long x, const uint8_t* alive) {
    return x != kRowTomb && (alive == nullptr || alive[static_cast<int32_t>(static_cast<uint32_t>(x))]);
}

struct CountLive {
    const unsigned long long* xpe;
    const uint8_t* alive;
    int64_t* deg;
    __device__ void operator()(const RowTask& t, int64_t e, bool in) const {
        const bool ok = in && entry_live(xpe[e], alive);
        const unsigned b = __ballot_sync(0xffffffffu, ok);
        if (lane_of() == 0 && b) atomicAdd(reinterpret_cast<unsigned long long*>(&deg[t.arg]),
                                           static_cast<unsigned long long>(__popc(b)));
    }
};

struct FillCsr {
    const unsigned long long* xpe;
    const uint8_t* alive;
    const int64_t* rp;
    int32_t* cursor;
    int32_t* col;
    int32_t* elab;
    __device__ void operator()(const RowTask& t, int64_t e, bool in) const {
        unsigned long long x = 0;
        bool ok = false;
        if (in) {
            x = xpe[e];
            ok = entry_live(x, alive);
        }
        const unsigned b = __ballot_sync(0xffffffffu, ok);
        if (b == 0u) return;
        int base = 0;
        if (lane_of() == 0) base = atomicAdd(&cursor[t.arg], __popc(b));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (ok) {
            const int64_t p = rp[t.arg] + base + __popc(b & ((1u << lane_of()) - 1u));
            col[p] = static_cast<int32_t>(static_cast<uint32_t>(x));
            elab[p] = static_cast<int32_t>(x >> 32);
        }
    }
};

StoreView store_view(bisim_ctx* ctx) {
    return StoreView{ctx->xro, ctx->xlen, ctx->xcap, ctx->xpe, ctx->yro, ctx->ylen, ctx->ycap, ctx->ype};
}

}  // namespace

void store_release(bisim_ctx* ctx, cudaStream_t s) {
    const size_t n = static_cast<size_t>(std::max(ctx->n, 1));
    ctx_free(ctx, ctx->xro, 8 * (n + 1), s);
    ctx_free(ctx, ctx->xlen, 4 * n, s);
    ctx_free(ctx, ctx->xcap, 4 * n, s);
    ctx_free(ctx, ctx->xpe, 8 * static_cast<size_t>(std::max<int64_t>(ctx->xpool, 1)), s);
    ctx_free(ctx, ctx->yro, 8 * (n + 1), s);
    ctx_free(ctx, ctx->ylen, 4 * n, s);
    ctx_free(ctx, ctx->ycap, 4 * n, s);
    ctx_free(ctx, ctx->ype, 4 * static_cast<size_t>(std::max<int64_t>(ctx->ypool, 1)), s);
    ctx_free(ctx, ctx->dtail, 8 * 4, s);
    ctx_free(ctx, ctx->addo, 4 * n, s);
    ctx_free(ctx, ctx->addi, 4 * n, s);
    ctx_free(ctx, ctx->xmark, 4 * n, s);
    ctx_free(ctx, ctx->dmark, 4 * (n / 32 + 1), s);
    ctx->xro = ctx->yro = ctx->dtail = nullptr;
    ctx->xlen = ctx->xcap = ctx->ylen = ctx->ycap = ctx->ype = ctx->addo = ctx->addi = nullptr;
    ctx->xmark = ctx->dmark = nullptr;
    ctx->xpe = nullptr;
    ctx->xpool = ctx->ypool = 0;
    ctx->store_ready = false;
}

bisim_status store_build(bisim_ctx* ctx, cudaStream_t s, int64_t room_out, int64_t room_in) {
    bisim_status st;
    if ((st = csr_from_store(ctx, s)) != BISIM_OK) return st;
    store_release(ctx, s);
    if ((st = ensure_edge_sources(ctx, s)) != BISIM_OK) return st;
    const int32_t n = ctx->n;
    const int64_t m = ctx->m;
    const size_t nn = static_cast<size_t>(std::max(n, 1));
    cudaError_t e;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->xro), 8 * (nn + 1), s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->xlen), 4 * nn, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->xcap), 4 * nn, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->yro), 8 * (nn + 1), s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->ylen), 4 * nn, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->ycap), 4 * nn, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dtail), 8 * 4, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->addo), 4 * nn, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->addi), 4 * nn, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->xmark), 4 * nn, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dmark), 4 * (nn / 32 + 1), s)))
        return cuda_error(ctx, e, "alloc row store");
    const size_t tw = scan_temp_words(static_cast<int64_t>(n) + 1);
    int64_t* scratch = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), 8 * (2 * (nn + 1) + tw), s)))
        return cuda_error(ctx, e, "alloc store scratch");
    int64_t* caps = scratch;
    int64_t* tmp = scratch + 2 * (nn + 1);
    BISIM_SITE(site, "store_build");
    cudaMemsetAsync(ctx->addo, 0, 4 * nn, s);
    cudaMemsetAsync(ctx->addi, 0, 4 * nn, s);
    cudaMemsetAsync(ctx->xmark, 0, 4 * nn, s);
    cudaMemsetAsync(ctx->dmark, 0, 4 * (nn / 32 + 1), s);
    cudaMemsetAsync(ctx->ylen, 0, 4 * nn, s);
    int64_t totals[2] = {0, 0};
    {
        Launch L(site, s, n, m, 24.0 * n + 4.0 * m);
        k_store_out_caps<<<grid_for(n + 1, 256), 256, 0, s>>>(ctx->row_ptr, n, ctx->xlen, ctx->xcap, caps);
        exclusive_scan_i64(caps, ctx->xro, n + 1, tmp, s);
        if (m > 0) k_store_in_degrees<<<grid_for(m, 256), 256, 0, s>>>(ctx->col, m, ctx->ylen);
        k_store_in_caps<<<grid_for(n + 1, 256), 256, 0, s>>>(n, ctx->ylen, ctx->ycap, caps + nn + 1);
        exclusive_scan_i64(caps + nn + 1, ctx->yro, n + 1, tmp, s);
    }
    cudaMemcpyAsync(&totals[0], ctx->xro + n, 8, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&totals[1], ctx->yro + n, 8, cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) {
        cudaFreeAsync(scratch, s);
        return cuda_error(ctx, e, "size row store");
    }
    // room for rows that outgrow their capacity before the next rebuild
    ctx->xpool = totals[0] + std::max<int64_t>(std::max<int64_t>(totals[0] / 4, 1 << 20), room_out);
    ctx->ypool = totals[1] + std::max<int64_t>(std::max<int64_t>(totals[1] / 4, 1 << 20), room_in);
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->xpe), 8 * static_cast<size_t>(ctx->xpool), s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->ype), 4 * static_cast<size_t>(ctx->ypool), s))) {
        cudaFreeAsync(scratch, s);
        return cuda_error(ctx, e, "alloc row pools");
    }
    {
        Launch L(site, s, 0, m, 40.0 * m);
        if (m > 0)
            k_store_fill<<<grid_for(m, 256), 256, 0, s>>>(ctx->row_ptr, ctx->esrc, ctx->col, ctx->elab, m,
                                                         store_view(ctx));
    }
    int64_t tails[4] = {totals[0], totals[1], 0, 0};
    cudaMemcpyAsync(ctx->dtail, tails, sizeof(tails), cudaMemcpyHostToDevice, s);
    cudaFreeAsync(scratch, s);
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "build row store");
    ctx->store_ready = true;
    ctx->csr_stale = false;
    ctx->stats.device_bytes = ctx->device_bytes;
    return BISIM_OK;
}

bisim_status csr_from_store(bisim_ctx* ctx, cudaStream_t s) {
    if (!ctx->csr_stale) return BISIM_OK;
    const int32_t n = ctx->n;
    const size_t nn = static_cast<size_t>(std::max(n, 1));
    cudaError_t e;
    const size_t tw = scan_temp_words(static_cast<int64_t>(n) + 1);
    // scratch: degrees and row offsets (n + 1 each), scan words, cursors, three task lists
    const size_t bytes = 8 * (2 * (nn + 1) + tw) + 4 * nn + 3 * sizeof(RowTask) * nn + 256;
    char* scratch = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), bytes, s))) return cuda_error(ctx, e, "alloc CSR rebuild");
    int64_t* deg = reinterpret_cast<int64_t*>(scratch);
    int64_t* rp = deg + (nn + 1);
    int64_t* tmp = rp + (nn + 1);
    int32_t* cursor = reinterpret_cast<int32_t*>(tmp + tw);
    RowTask* tasks = reinterpret_cast<RowTask*>(reinterpret_cast<char*>(cursor) + ((4 * nn + 15) & ~size_t(15)));
    unsigned* tcnt = reinterpret_cast<unsigned*>(tasks + 3 * nn);
    TierLists TL{{tasks, tasks + nn, tasks + 2 * nn}, tcnt};
    cudaMemsetAsync(deg, 0, 8 * (nn + 1), s);
    cudaMemsetAsync(cursor, 0, 4 * nn, s);
    cudaMemsetAsync(tcnt, 0, 16, s);
    BISIM_SITE(site, "csr_from_store");
    {
        Launch L(site, s, n, 0, 24.0 * n);
        if (n > 0) k_store_row_tasks<<<grid_for(n, 256), 256, 0, s>>>(n, ctx->alive, store_view(ctx), TL);
        run_tiers(TL, CountLive{ctx->xpe, ctx->alive, deg}, s);
        exclusive_scan_i64(deg, rp, n + 1, tmp, s);
    }
    int64_t m = 0;
    cudaMemcpyAsync(&m, rp + n, 8, cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) {
        cudaFreeAsync(scratch, s);
        return cuda_error(ctx, e, "count store rows");
    }
    ctx_free(ctx, ctx->col, 4 * static_cast<size_t>(std::max<int64_t>(ctx->m, 1)), s);
    ctx_free(ctx, ctx->elab, 4 * static_cast<size_t>(std::max<int64_t>(ctx->m, 1)), s);
    ctx_free(ctx, ctx->esrc, 4 * static_cast<size_t>(std::max<int64_t>(ctx->esrc_cap, 1)), s);
    ctx->col = ctx->elab = ctx->esrc = nullptr;
    ctx->esrc_cap = 0;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->col), 4 * static_cast<size_t>(std::max<int64_t>(m, 1)), s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->elab), 4 * static_cast<size_t>(std::max<int64_t>(m, 1)), s))) {
        cudaFreeAsync(scratch, s);
        return cuda_error(ctx, e, "alloc CSR");
    }
    {
        Launch L(site, s, n, m, 16.0 * m);
        cudaMemcpyAsync(ctx->row_ptr, rp, 8 * (static_cast<size_t>(n) + 1), cudaMemcpyDeviceToDevice, s);
        run_tiers(TL, FillCsr{ctx->xpe, ctx->alive, ctx->row_ptr, cursor, ctx->col, ctx->elab}, s);
    }
    cudaFreeAsync(scratch, s);
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "rebuild CSR from the store");
    ctx->m = m;
    ctx->stats.n_edges = m;
    ctx->csr_stale = false;
    ctx->dense_ready = false;
    ctx->stats.device_bytes = ctx->device_bytes;
    return BISIM_OK;
}

}  // namespace bisim
