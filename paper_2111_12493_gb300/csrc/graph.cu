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

// Checks every edge and counts out-degrees (one atomic per distinct source in
// a warp; edge lists are often grouped by source). Degrees of a list that fails
// the check are never used.
__global__ void k_validate_coo(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                               int64_t m, int32_t n, const uint8_t* __restrict__ alive,
                               int32_t* __restrict__ deg, unsigned* err) {
    // trip count is uniform across the warp so the match below sees every lane
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; e0 < m; e0 += stride) {
        const int64_t e = e0 + threadIdx.x;
        int32_t s = -1;
        if (e < m) {
            s = src[e];
            const int32_t d = dst[e];
            bool ok = s >= 0 && s < n && d >= 0 && d < n;
            if (ok && alive != nullptr) ok = alive[s] && alive[d];
            if (!ok) {
                atomicOr(err, kErrBadInput);
                s = -1;
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, s);
        if (s >= 0 && (threadIdx.x & 31) == static_cast<unsigned>(__ffs(peers) - 1)) atomicAdd(&deg[s], __popc(peers));
    }
}

// Every edge written into its source's packed row of the layout: the row of
// position p is [prp[p], prp[p+1]); a per-row cursor hands out the slots, one
// atomic per distinct source in a warp (the lanes of one source take
// consecutive slots in lane order). Signatures are sets, so the order of the
// edges inside a row is never read; it follows the order in which warps reach
// the row's cursor. Edge lists grouped by source (the common case) write each
// row in runs.
__global__ void k_place_coo(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                            const int32_t* __restrict__ elab, int64_t m, const int32_t* __restrict__ vpos,
                            const int64_t* __restrict__ prp, int32_t* __restrict__ cursor,
                            unsigned long long* __restrict__ pe) {
    const unsigned lane = threadIdx.x & 31u;
    // trip count is uniform across the warp so the match below sees every lane
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; e0 < m; e0 += stride) {
        const int64_t e = e0 + threadIdx.x;
        int32_t pos = -1;
        if (e < m) pos = vpos[src[e]];
        const unsigned peers = __match_any_sync(0xffffffffu, pos);
        const int leader = __ffs(peers) - 1;
        int32_t base = 0;
        if (pos >= 0 && lane == static_cast<unsigned>(leader)) base = atomicAdd(&cursor[pos], __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (pos >= 0) {
            const int32_t r = base + __popc(peers & ((1u << lane) - 1u));
            pe[prp[pos] + r] = (static_cast<unsigned long long>(static_cast<uint32_t>(elab[e])) << 32) |
                               static_cast<uint32_t>(dst[e]);
        }
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
                            const int32_t* elab, cudaStream_t s) {
    const int32_t n = ctx->n;
    const int64_t m = ctx->m;
    const int64_t cap = std::max<int64_t>(m, 1);
    cudaError_t e;
    // scratch: out-degrees, then the per-row cursors of the placement
    const size_t nv = static_cast<size_t>(n) + 1;
    const size_t bytes = 2 * ((sizeof(int32_t) * nv + 255) & ~size_t(255));
    char* base = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&base), bytes, s))) return cuda_error(ctx, e, "alloc CSR scratch");
    int32_t* deg = reinterpret_cast<int32_t*>(base);
    int32_t* cursor = reinterpret_cast<int32_t*>(base + bytes / 2);
    unsigned long long* rows = nullptr;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&rows), sizeof(unsigned long long) * cap, s))) {
        cudaFreeAsync(base, s);
        return cuda_error(ctx, e, "alloc packed rows");
    }

    cudaMemsetAsync(&ctx->dstate->error, 0, sizeof(unsigned), s);
    cudaMemsetAsync(deg, 0, sizeof(int32_t) * (n + 1), s);
    BISIM_SITE(site_val, "validate_edges");
    BISIM_SITE(site_pack, "csr_place");
    if (m > 0)
        Launch(site_val, s, 0, m, 8.0 * m),
        k_validate_coo<<<grid_for(std::min<int64_t>(m, 1 << 22), 256), 256, 0, s>>>(src, dst, m, n, ctx->alive, deg,
                                                                                   &ctx->dstate->error);
    cudaMemcpyAsync(ctx->hstate, ctx->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) { cudaFreeAsync(base, s); return cuda_error(ctx, e, "validate edges"); }
    if (ctx->hstate->error & kErrBadInput) {
        cudaFreeAsync(base, s);
        return set_error(ctx, BISIM_EINVAL, "edge endpoint out of range [0, n) or on a dead vertex");
    }
    bisim_status st = dense_layout_positions(ctx, deg, s);
    if (st != BISIM_OK) {
        cudaFreeAsync(base, s);
        return st;
    }
    if (m > 0) {
        // read src, dst, label, the source's position and row offset; write the packed word
        cudaMemsetAsync(cursor, 0, sizeof(int32_t) * nv, s);
        Launch L(site_pack, s, 0, m, 24.0 * m);
        k_place_coo<<<grid_for(std::min<int64_t>(m, 1 << 22), 256), 256, 0, s>>>(src, dst, elab, m, ctx->dvpos,
                                                                                 ctx->dprp, cursor, rows);
    }
    ctx_free(ctx, ctx->dpe, sizeof(unsigned long long) * ctx->dpe_cap, s);
    ctx->dpe = rows;
    ctx->dpe_cap = cap;
    cudaFreeAsync(base, s);
    if ((e = cudaGetLastError())) return cuda_error(ctx, e, "build layout");
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
