// Out-CSR construction, validation and degree bucketing.
#include <algorithm>

#include "common.cuh"
#include "prof.cuh"

namespace bisim {

namespace {

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
unsigned grid_for(int64_t n, int threads) {
    return static_cast<unsigned>(std::max<int64_t>(1, cdiv(n, threads)));
}

// Runs of equal keys among a warp's lanes (lane order): a lane heads a run
// when its key differs from the previous lane's. Sources grouped in the edge
// list give a few runs per warp; any order stays correct, with more runs.
__device__ __forceinline__ unsigned run_heads(int32_t key, unsigned lane) {
    const int32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    return __ballot_sync(0xffffffffu, lane == 0 || prev != key);
}

// Lanes in the run headed by `lane` (a head): up to the next head.
__device__ __forceinline__ int run_length(unsigned heads, unsigned lane) {
    const unsigned after = lane == 31 ? 0u : heads >> (lane + 1);
    return after ? __ffs(after) : 32 - static_cast<int>(lane);
}

// The head of the run that holds `lane`.
__device__ __forceinline__ int run_head(unsigned heads, unsigned lane) {
    const unsigned upto = lane == 31 ? heads : heads & ((2u << lane) - 1u);
    return 31 - __clz(upto);
}

// Checks every edge (or, with dst null, every source; k_validate_dst then
// checks the targets), and finds out whether the list is sorted by source. For
// a sorted list each source's edges form one run [start, end) of the list:
// the run's first edge records start[v] and adds -start to deg[v], its last
// edge adds end, so deg[v] = end - start (in modular 32-bit arithmetic, exact
// for any degree below 2^32) with two atomics per vertex on distinct
// addresses. For an unsorted list these values are not used (k_count_coo
// counts again). A list that fails the check is not used at all.
__global__ void __launch_bounds__(256) k_validate_coo(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                                      int64_t m, int32_t n, const uint8_t* __restrict__ alive,
                                                      uint32_t* __restrict__ deg, int64_t* __restrict__ start,
                                                      DevState* st) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t s = src[e];
        const int32_t d = dst != nullptr ? dst[e] : 0;
        const int32_t prev = e > 0 ? src[e - 1] : -1;
        const int32_t next = e + 1 < m ? src[e + 1] : -1;
        bool ok = s >= 0 && s < n && d >= 0 && d < n;
        if (ok && alive != nullptr) ok = alive[s] && (dst == nullptr || alive[d]);
        if (!ok) {
            atomicOr(&st->error, kErrBadInput);
            continue;
        }
        if (prev > s) atomicOr(&st->unsorted, 1u);
        if (prev != s) {
            start[s] = e;
            atomicAdd(&deg[s], 0u - static_cast<uint32_t>(e));
        }
        if (next != s) atomicAdd(&deg[s], static_cast<uint32_t>(e + 1));
    }
}

// The targets' check of a list whose sources k_validate_coo checked alone.
__global__ void __launch_bounds__(256) k_validate_dst(const int32_t* __restrict__ dst, int64_t m, int32_t n,
                                                      const uint8_t* __restrict__ alive, DevState* st) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t d = dst[e];
        if (d < 0 || d >= n || (alive != nullptr && !alive[d])) atomicOr(&st->error, kErrBadInput);
    }
}

// Out-degrees of an unsorted list: one atomic per run of equal sources in a
// warp.
__global__ void __launch_bounds__(256) k_count_coo(const int32_t* __restrict__ src, int64_t m,
                                                   uint32_t* __restrict__ deg) {
    const unsigned lane = threadIdx.x & 31u;
    // trip count is uniform across the warp so the shuffles see every lane
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; e0 < m; e0 += stride) {
        const int64_t e = e0 + threadIdx.x;
        const int32_t s = e < m ? src[e] : -1;
        const unsigned heads = run_heads(s, lane);
        if (s >= 0 && ((heads >> lane) & 1u)) atomicAdd(&deg[s], static_cast<uint32_t>(run_length(heads, lane)));
    }
}

__device__ __forceinline__ unsigned long long pack_word(int32_t label, int32_t target) {
    return (static_cast<unsigned long long>(static_cast<uint32_t>(label)) << 32) | static_cast<uint32_t>(target);
}

// Every edge written into its source's packed row of the layout: the row of
// position p is [prp[p], prp[p+1]). A sorted list places edge e at offset
// e - start[v] of its row: no atomics, and the row keeps the list's order.
__global__ void __launch_bounds__(256) k_place_sorted(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                                      const int32_t* __restrict__ elab, int64_t m,
                                                      const int32_t* __restrict__ vpos, const int64_t* __restrict__ prp,
                                                      const int64_t* __restrict__ start,
                                                      unsigned long long* __restrict__ pe) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t v = src[e];
        pe[prp[vpos[v]] + (e - start[v])] = pack_word(elab[e], dst[e]);
    }
}

// The same for an unsorted list: a per-row cursor hands out the slots, one
// atomic per run of equal sources in a warp (the run's lanes take consecutive
// slots in lane order). Signatures are sets, so the order of the edges inside
// a row is never read; it follows the order in which warps reach the row's
// cursor.
__global__ void __launch_bounds__(256) k_place_coo(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                                   const int32_t* __restrict__ elab, int64_t m,
                                                   const int32_t* __restrict__ vpos, const int64_t* __restrict__ prp,
                                                   int32_t* __restrict__ cursor, unsigned long long* __restrict__ pe) {
    const unsigned lane = threadIdx.x & 31u;
    // trip count is uniform across the warp so the shuffles see every lane
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; e0 < m; e0 += stride) {
        const int64_t e = e0 + threadIdx.x;
        const int32_t pos = e < m ? vpos[src[e]] : -1;
        const unsigned heads = run_heads(pos, lane);
        int32_t base = 0;
        if (pos >= 0 && ((heads >> lane) & 1u)) base = atomicAdd(&cursor[pos], run_length(heads, lane));
        const int h = run_head(heads, lane);
        base = __shfl_sync(0xffffffffu, base, h);
        if (pos >= 0) pe[prp[pos] + base + (static_cast<int>(lane) - h)] = pack_word(elab[e], dst[e]);
    }
}

__global__ void k_validate_csr(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               int32_t n, int64_t m, const uint8_t* __restrict__ alive,
                               unsigned* err) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int64_t v = t0; v <= n; v += stride) {
        int64_t a = rp[v];
        bool ok = a >= 0 && a <= m;
        if (v == 0) ok = ok && a == 0;
        if (v == n) ok = ok && a == m;
        if (v < n) {
            int64_t b = rp[v + 1];
            ok = ok && b >= a;
            if (alive != nullptr && !alive[v]) ok = ok && b == a;
        }
        if (!ok) atomicOr(err, kErrBadInput);
    }
    for (int64_t e = t0; e < m; e += stride) {
        int32_t d = col[e];
        bool ok = d >= 0 && d < n;
        if (ok && alive != nullptr) ok = alive[d];
        if (!ok) atomicOr(err, kErrBadInput);
    }
}

}  // namespace

// COO -> the round layout directly: out-degrees, then the positions of the
// layout (vertices grouped by degree class) and their row offsets, then every
// edge placed into its source's row (k_place_coo). The (label, target) words
// are the layout's packed rows; the vertex-ordered CSR is rebuilt from them
// only if an update or the list-mode path asks for it.
bisim_status build_from_coo(bisim_ctx* ctx, const int32_t* src, const int32_t* dst,
                            const int32_t* elab, cudaStream_t s, const CooArrival* arrival) {
    const int32_t n = ctx->n;
    const int64_t m = ctx->m;
    const int64_t cap = std::max<int64_t>(m, 1);
    cudaError_t e;
    // scratch: out-degrees, then the runs' first edges (sorted list) or the
    // per-row cursors (unsorted list)
    const size_t nv = static_cast<size_t>(n) + 1;
    const size_t deg_bytes = (sizeof(uint32_t) * nv + 255) & ~size_t(255);
    const size_t bytes = deg_bytes + sizeof(int64_t) * nv;
    char* base = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&base), bytes, s))) return cuda_error(ctx, e, "alloc CSR scratch");
    uint32_t* deg = reinterpret_cast<uint32_t*>(base);
    int64_t* start = reinterpret_cast<int64_t*>(base + deg_bytes);
    int32_t* cursor = reinterpret_cast<int32_t*>(start);
    unsigned long long* rows = nullptr;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&rows), sizeof(unsigned long long) * cap, s))) {
        cudaFreeAsync(base, s);
        return cuda_error(ctx, e, "alloc packed rows");
    }

    cudaMemsetAsync(&ctx->dstate->error, 0, sizeof(unsigned), s);
    cudaMemsetAsync(&ctx->dstate->unsorted, 0, sizeof(unsigned), s);
    cudaMemsetAsync(deg, 0, sizeof(uint32_t) * nv, s);
    BISIM_SITE(site_val, "validate_edges");
    BISIM_SITE(site_cnt, "count_edges");
    BISIM_SITE(site_pack, "csr_place");
    const unsigned grid = grid_for(std::min<int64_t>(m, 1 << 22), 256);
    // arriving arrays: the sources are checked and counted while the targets
    // and labels are still being copied in
    if (arrival != nullptr) cudaStreamWaitEvent(s, arrival->src, 0);
    if (m > 0)
        Launch(site_val, s, 0, m, arrival ? 4.0 * m : 8.0 * m),
        k_validate_coo<<<grid, 256, 0, s>>>(src, arrival ? nullptr : dst, m, n, ctx->alive, deg, start, ctx->dstate);
    cudaMemcpyAsync(ctx->hstate, ctx->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) { cudaFreeAsync(base, s); return cuda_error(ctx, e, "validate edges"); }
    if (ctx->hstate->error & kErrBadInput) {
        cudaFreeAsync(base, s);
        return set_error(ctx, BISIM_EINVAL, "edge endpoint out of range [0, n) or on a dead vertex");
    }
    const bool sorted = ctx->hstate->unsorted == 0;
    if (!sorted && m > 0) {
        cudaMemsetAsync(deg, 0, sizeof(uint32_t) * nv, s);
        Launch(site_cnt, s, 0, m, 4.0 * m),
        k_count_coo<<<grid, 256, 0, s>>>(src, m, deg);
    }
    bisim_status st = dense_layout_positions(ctx, reinterpret_cast<const int32_t*>(deg), s);
    if (st != BISIM_OK) {
        cudaFreeAsync(base, s);
        return st;
    }
    if (arrival != nullptr && m > 0) {
        cudaStreamWaitEvent(s, arrival->dst, 0);
        {
            Launch L(site_val, s, 0, m, 4.0 * m);
            k_validate_dst<<<grid, 256, 0, s>>>(dst, m, n, ctx->alive, ctx->dstate);
        }
        cudaStreamWaitEvent(s, arrival->lab, 0);
        if (arrival->arrived != nullptr) {
            // the host link is free again: let the next upload start
            if ((e = cudaEventSynchronize(arrival->lab))) {
                cudaFreeAsync(base, s);
                return cuda_error(ctx, e, "edge labels copy");
            }
            arrival->arrived(arrival->arrived_arg);
        }
    }
    if (m > 0) {
        // read src, dst, label, the source's position and row offset; write the packed word
        Launch L(site_pack, s, 0, m, 24.0 * m);
        if (sorted) {
            k_place_sorted<<<grid, 256, 0, s>>>(src, dst, elab, m, ctx->dvpos, ctx->dprp, start, rows);
        } else {
            cudaMemsetAsync(cursor, 0, sizeof(int32_t) * nv, s);
            k_place_coo<<<grid, 256, 0, s>>>(src, dst, elab, m, ctx->dvpos, ctx->dprp, cursor, rows);
        }
    }
    ctx_free(ctx, ctx->dpe, sizeof(unsigned long long) * ctx->dpe_cap, s);
    ctx->dpe = rows;
    ctx->dpe_cap = cap;
    cudaFreeAsync(base, s);
    if ((e = cudaGetLastError())) return cuda_error(ctx, e, "build layout");
    if (arrival != nullptr && m > 0) {
        // the targets' check ran after the layout was made: read it now
        cudaMemcpyAsync(ctx->hstate, ctx->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "validate edge targets");
        if (ctx->hstate->error & kErrBadInput)
            return set_error(ctx, BISIM_EINVAL, "edge endpoint out of range [0, n) or on a dead vertex");
    }
    return dense_layout_hubs(ctx, false, s);
}

bisim_status build_from_csr(bisim_ctx* ctx, const int64_t* row_ptr, const int32_t* col,
                            const int32_t* elab, cudaStream_t s) {
    const int32_t n = ctx->n;
    const int64_t m = ctx->m;
    cudaError_t e;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->row_ptr), sizeof(int64_t) * (n + 1), s))) return cuda_error(ctx, e, "alloc row_ptr");
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->col), sizeof(int32_t) * std::max<int64_t>(m, 1), s))) return cuda_error(ctx, e, "alloc col");
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->elab), sizeof(int32_t) * std::max<int64_t>(m, 1), s))) return cuda_error(ctx, e, "alloc elab");
    cudaMemcpyAsync(ctx->row_ptr, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDefault, s);
    if (m > 0) {
        cudaMemcpyAsync(ctx->col, col, sizeof(int32_t) * m, cudaMemcpyDefault, s);
        cudaMemcpyAsync(ctx->elab, elab, sizeof(int32_t) * m, cudaMemcpyDefault, s);
    }
    cudaMemsetAsync(&ctx->dstate->error, 0, sizeof(unsigned), s);
    BISIM_SITE(site_vcsr, "validate_csr");
    Launch(site_vcsr, s, n + 1, m, 8.0 * (n + 1) + 4.0 * m),
    k_validate_csr<<<grid_for(std::min<int64_t>(std::max<int64_t>(m, n + 1), 1 << 22), 256), 256, 0, s>>>(
        ctx->row_ptr, ctx->col, n, m, ctx->alive, &ctx->dstate->error);
    cudaMemcpyAsync(ctx->hstate, ctx->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "validate CSR");
    if (ctx->hstate->error & kErrBadInput)
        return set_error(ctx, BISIM_EINVAL, "malformed CSR: row_ptr not a prefix sum of [0, m], a target out of range, or an edge on a dead vertex");
    return BISIM_OK;
}

}  // namespace bisim
