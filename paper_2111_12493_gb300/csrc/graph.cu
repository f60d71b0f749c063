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

// Sort keys are the sources' positions in the layout (so the sorted edges are
// its packed rows); values are the packed (label, target) words.
__global__ void k_pack_coo(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                           const int32_t* __restrict__ elab, int64_t m, const int32_t* __restrict__ vpos,
                           uint32_t* __restrict__ keys, uint64_t* __restrict__ vals) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        keys[e] = static_cast<uint32_t>(vpos[src[e]]);
        vals[e] = (static_cast<uint64_t>(static_cast<uint32_t>(elab[e])) << 32) | static_cast<uint32_t>(dst[e]);
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

// Degree class of each live vertex (see kNumClasses); dead vertices get kClassDead.
__global__ void k_classify(const int64_t* __restrict__ rp, const uint8_t* __restrict__ alive,
                           int32_t n, int small_max, int mid_max, uint32_t* __restrict__ keys,
                           uint64_t* __restrict__ vals) {
    int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int64_t d = rp[v + 1] - rp[v];
    uint32_t c;
    if (alive != nullptr && !alive[v]) {
        c = kClassDead;
    } else if (d <= small_max || d == 0) {
        c = d <= 4 ? 0u : d <= 8 ? 1u : d <= 16 ? 2u : 3u;
    } else if (d <= mid_max) {
        int lg = 64 - __clzll(static_cast<unsigned long long>(d - 1));   // ceil(log2 d)
        lg = lg < 6 ? 6 : lg;
        c = static_cast<uint32_t>(kSmallClasses + (lg - 6));
    } else {
        c = kClassHub;
    }
    keys[v] = c;
    vals[v] = static_cast<uint64_t>(v);
}

__global__ void k_class_bounds(const uint32_t* __restrict__ sorted_cls, int32_t n,
                               int64_t* __restrict__ begin) {
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // dead vertices (kClassDead) sort last and map to the end marker kNumClasses
    int c = static_cast<int>(min(sorted_cls[i], static_cast<uint32_t>(kNumClasses)));
    int p = i == 0 ? -1 : static_cast<int>(min(sorted_cls[i - 1], static_cast<uint32_t>(kNumClasses)));
    // first vertex of class c; empty classes between p and c start here too
    for (int q = p + 1; q <= c; ++q) begin[q] = i;
}

__global__ void k_class_edges(const uint32_t* __restrict__ sorted_cls, const uint64_t* __restrict__ sorted_v,
                              const int64_t* __restrict__ rp, int32_t n, unsigned long long* __restrict__ out) {
    __shared__ unsigned long long acc[kNumClasses];
    if (threadIdx.x < kNumClasses) acc[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    uint32_t c = kNumClasses;
    unsigned long long d = 0;
    if (i < n) {
        c = min(sorted_cls[i], static_cast<uint32_t>(kNumClasses));
        if (c < kNumClasses) {
            const int64_t v = static_cast<int64_t>(sorted_v[i]);
            d = static_cast<unsigned long long>(rp[v + 1] - rp[v]);
        }
    }
    // classes are sorted, so a warp holds one or two of them: reduce per class first
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    unsigned long long tot = d;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_down_sync(0xffffffffu, tot, o);
        const int src = static_cast<int>(threadIdx.x & 31) + o;
        if (src < 32 && ((peers >> src) & 1u)) tot += y;
    }
    if (c < kNumClasses && (threadIdx.x & 31) == static_cast<unsigned>(__ffs(peers) - 1)) atomicAdd(&acc[c], tot);
    __syncthreads();
    if (threadIdx.x < kNumClasses && acc[threadIdx.x]) atomicAdd(&out[threadIdx.x], acc[threadIdx.x]);
}

__global__ void k_take_low(const uint64_t* __restrict__ vals, int64_t n, int32_t* __restrict__ out) {
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = static_cast<int32_t>(vals[i]);
}

// Row bounds [row_ptr[v], row_ptr[v + 1]) of the listed hubs, interleaved.
__global__ void k_hub_bounds(const int32_t* __restrict__ hubs, int64_t nh, const int64_t* __restrict__ rp,
                             int64_t* __restrict__ out) {
    const int64_t h = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (h >= nh) return;
    out[2 * h] = rp[hubs[h]];
    out[2 * h + 1] = rp[hubs[h] + 1];
}

int bits_for(int64_t n) {
    int b = 0;
    while ((static_cast<int64_t>(1) << b) < n) ++b;
    return b;
}

}  // namespace

// COO -> the round layout directly: out-degrees, then the positions of the
// layout (vertices grouped by degree class), then one stable LSD radix sort of
// the edges keyed by their source's position. The sorted (label, target)
// words are the layout's packed rows; the vertex-ordered CSR is rebuilt from
// them only if an update or the list-mode path asks for it.
bisim_status build_from_coo(bisim_ctx* ctx, const int32_t* src, const int32_t* dst,
                            const int32_t* elab, cudaStream_t s) {
    const int32_t n = ctx->n;
    const int64_t m = ctx->m;
    const int64_t cap = std::max<int64_t>(m, 1);
    cudaError_t e;
    const size_t tmp_words = std::max(radix_temp_words(m), scan_temp_words(n + 1));
    const size_t bytes = sizeof(uint32_t) * 2 * cap + sizeof(int32_t) * (n + 1) + sizeof(int64_t) * tmp_words + 256 * 4;
    char* scratch = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), bytes, s))) return cuda_error(ctx, e, "alloc CSR scratch");
    auto carve = [&](size_t b) { char* p = scratch; scratch += (b + 255) & ~size_t(255); return p; };
    char* base = scratch;
    uint32_t* k0 = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * cap));
    uint32_t* k1 = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * cap));
    int32_t* deg = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * (n + 1)));
    int64_t* tmp = reinterpret_cast<int64_t*>(carve(sizeof(int64_t) * tmp_words));
    uint64_t *v0 = nullptr, *v1 = nullptr;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&v0), sizeof(uint64_t) * cap, s)) ||
        (e = ctx_alloc(ctx, reinterpret_cast<void**>(&v1), sizeof(uint64_t) * cap, s))) {
        cudaFreeAsync(base, s);
        return cuda_error(ctx, e, "alloc packed rows");
    }

    cudaMemsetAsync(&ctx->dstate->error, 0, sizeof(unsigned), s);
    cudaMemsetAsync(deg, 0, sizeof(int32_t) * (n + 1), s);
    BISIM_SITE(site_val, "validate_edges");
    BISIM_SITE(site_pack, "csr_pack");
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
    int which = 0;
    if (m > 0) {
        {
            // read src, dst, label and the source's position; write key + value
            Launch L(site_pack, s, 0, m, 28.0 * m);
            k_pack_coo<<<grid_for(std::min<int64_t>(m, 1 << 22), 256), 256, 0, s>>>(src, dst, elab, m, ctx->dvpos, k0,
                                                                                    v0);
        }
        which = radix_sort_pairs(k0, v0, k1, v1, m, bits_for(n), tmp, s);
    }
    uint64_t* rows = which ? v1 : v0;
    ctx_free(ctx, which ? v0 : v1, sizeof(uint64_t) * cap, s);
    ctx_free(ctx, ctx->dpe, sizeof(unsigned long long) * ctx->dpe_cap, s);
    ctx->dpe = reinterpret_cast<unsigned long long*>(rows);
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

bisim_status ensure_buckets(bisim_ctx* ctx, cudaStream_t s) {
    if (ctx->buckets_ready) return BISIM_OK;
    bisim_status st = ensure_vertex_csr(ctx, s);
    if (st != BISIM_OK) return st;
    st = build_buckets(ctx, s);
    if (st == BISIM_OK) ctx->buckets_ready = true;
    return st;
}

bisim_status build_buckets(bisim_ctx* ctx, cudaStream_t s) {
    const int32_t n = ctx->n;
    cudaError_t e;
    // a rebuild after the graph changed: release the previous layout
    ctx_free(ctx, ctx->class_list, sizeof(int32_t) * std::max(n, 1), s);
    ctx_free(ctx, ctx->chunks, sizeof(HubChunk) * ctx->n_chunks, s);
    ctx_free(ctx, ctx->hub_toff, sizeof(int64_t) * ctx->n_hub, s);
    ctx_free(ctx, ctx->hub_tmask, sizeof(uint32_t) * ctx->n_hub, s);
    ctx_free(ctx, ctx->hub_tab, sizeof(unsigned long long) * ctx->hub_tab_words, s);
    ctx_free(ctx, ctx->hub_acc, sizeof(HubAcc) * ctx->n_hub, s);
    ctx->class_list = nullptr;
    ctx->chunks = nullptr;
    ctx->hub_toff = nullptr;
    ctx->hub_tmask = nullptr;
    ctx->hub_tab = nullptr;
    ctx->hub_acc = nullptr;
    ctx->n_chunks = 0;
    ctx->n_hub = 0;
    ctx->hub_tab_words = 0;
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->class_list), sizeof(int32_t) * std::max(n, 1), s))) return cuda_error(ctx, e, "alloc class list");
    const size_t tmp_words = radix_temp_words(n);
    char* scratch = nullptr;
    const size_t bytes = (sizeof(uint32_t) * 2 + sizeof(uint64_t) * 2) * std::max(n, 1) + sizeof(int64_t) * (tmp_words + 2 * kNumClasses + 1) + 8 * 256;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), bytes, s))) return cuda_error(ctx, e, "alloc bucket scratch");
    char* base = scratch;
    auto carve = [&](size_t b) { char* p = scratch; scratch += (b + 255) & ~size_t(255); return p; };
    uint32_t* k0 = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * std::max(n, 1)));
    uint32_t* k1 = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * std::max(n, 1)));
    uint64_t* v0 = reinterpret_cast<uint64_t*>(carve(sizeof(uint64_t) * std::max(n, 1)));
    uint64_t* v1 = reinterpret_cast<uint64_t*>(carve(sizeof(uint64_t) * std::max(n, 1)));
    int64_t* tmp = reinterpret_cast<int64_t*>(carve(sizeof(int64_t) * tmp_words));
    int64_t* dbegin = reinterpret_cast<int64_t*>(carve(sizeof(int64_t) * (kNumClasses + 1)));
    unsigned long long* dedges = reinterpret_cast<unsigned long long*>(carve(sizeof(unsigned long long) * kNumClasses));
    cudaMemsetAsync(dedges, 0, sizeof(unsigned long long) * kNumClasses, s);

    int64_t begin[kNumClasses + 1];
    for (int c = 0; c <= kNumClasses; ++c) begin[c] = n;
    cudaMemcpyAsync(dbegin, begin, sizeof(begin), cudaMemcpyHostToDevice, s);
    if (n > 0) {
        BISIM_SITE(site, "bucket_vertices");
        {
            Launch L(site, s, n, 0, 8.0 * n + 12.0 * n);
            k_classify<<<grid_for(n, 256), 256, 0, s>>>(ctx->row_ptr, ctx->alive, n, ctx->opt.small_max_degree,
                                                       ctx->opt.mid_max_degree, k0, v0);
        }
        int which = radix_sort_pairs(k0, v0, k1, v1, n, 8, tmp, s);
        const uint32_t* sk = which ? k1 : k0;
        const uint64_t* sv = which ? v1 : v0;
        Launch L(site, s, n, 0, 36.0 * n);
        k_class_bounds<<<grid_for(n, 256), 256, 0, s>>>(sk, n, dbegin);
        k_class_edges<<<grid_for(n, 256), 256, 0, s>>>(sk, sv, ctx->row_ptr, n, dedges);
        k_take_low<<<grid_for(n, 256), 256, 0, s>>>(sv, n, ctx->class_list);
    }
    unsigned long long cedges[kNumClasses];
    cudaMemcpyAsync(cedges, dedges, sizeof(cedges), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(begin, dbegin, sizeof(begin), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) { cudaFreeAsync(base, s); return cuda_error(ctx, e, "bucket vertices"); }
    cudaFreeAsync(base, s);
    // classes absent at the tail start where the next present one starts
    for (int c = kNumClasses - 1; c >= 0; --c) begin[c] = std::min(begin[c], begin[c + 1]);
    for (int c = 0; c <= kNumClasses; ++c) ctx->class_begin[c] = begin[c];
    for (int c = 0; c < kNumClasses; ++c) ctx->class_edges[c] = static_cast<int64_t>(cedges[c]);
    ctx->hub_list = ctx->class_list + begin[kClassHub];
    ctx->n_hub = begin[kClassHub + 1] - begin[kClassHub];

    // hub chunks and dedup tables (host-side layout; the hub count is small)
    if (ctx->n_hub > 0) {
        std::vector<int32_t> hubs(ctx->n_hub);
        std::vector<int64_t> bounds(2 * ctx->n_hub);
        int64_t* dbounds = nullptr;
        if ((e = cudaMallocAsync(reinterpret_cast<void**>(&dbounds), sizeof(int64_t) * 2 * ctx->n_hub, s)))
            return cuda_error(ctx, e, "alloc hub bounds");
        k_hub_bounds<<<grid_for(ctx->n_hub, 256), 256, 0, s>>>(ctx->hub_list, ctx->n_hub, ctx->row_ptr, dbounds);
        cudaMemcpyAsync(hubs.data(), ctx->hub_list, sizeof(int32_t) * ctx->n_hub, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(bounds.data(), dbounds, sizeof(int64_t) * 2 * ctx->n_hub, cudaMemcpyDeviceToHost, s);
        cudaFreeAsync(dbounds, s);
        if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "read hub rows");
        std::vector<int64_t> rb(ctx->n_hub), re(ctx->n_hub);
        for (int64_t h = 0; h < ctx->n_hub; ++h) {
            rb[h] = bounds[2 * h];
            re[h] = bounds[2 * h + 1];
        }
        std::vector<HubChunk> chunks;
        std::vector<int64_t> toff(ctx->n_hub);
        std::vector<uint32_t> tmask(ctx->n_hub);
        int64_t words = 0;
        const int64_t csz = std::max(256, ctx->opt.hub_chunk);
        for (int64_t h = 0; h < ctx->n_hub; ++h) {
            int64_t d = re[h] - rb[h];
            uint64_t sz = 64;
            while (sz < static_cast<uint64_t>(2 * d)) sz <<= 1;
            toff[h] = words;
            tmask[h] = static_cast<uint32_t>(sz - 1);
            words += static_cast<int64_t>(sz);
            for (int64_t b = rb[h]; b < re[h]; b += csz)
                chunks.push_back(HubChunk{static_cast<int32_t>(h), hubs[h], b, std::min(re[h], b + csz)});
        }
        ctx->n_chunks = static_cast<int64_t>(chunks.size());
        ctx->hub_tab_words = words;
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->chunks), sizeof(HubChunk) * chunks.size(), s))) return cuda_error(ctx, e, "alloc hub chunks");
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->hub_toff), sizeof(int64_t) * ctx->n_hub, s))) return cuda_error(ctx, e, "alloc hub offsets");
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->hub_tmask), sizeof(uint32_t) * ctx->n_hub, s))) return cuda_error(ctx, e, "alloc hub masks");
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->hub_tab), sizeof(unsigned long long) * words, s))) return cuda_error(ctx, e, "alloc hub tables");
        if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->hub_acc), sizeof(HubAcc) * ctx->n_hub, s))) return cuda_error(ctx, e, "alloc hub accumulators");
        cudaMemcpyAsync(ctx->chunks, chunks.data(), sizeof(HubChunk) * chunks.size(), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(ctx->hub_toff, toff.data(), sizeof(int64_t) * ctx->n_hub, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(ctx->hub_tmask, tmask.data(), sizeof(uint32_t) * ctx->n_hub, cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(ctx->hub_tab, 0, sizeof(unsigned long long) * words, s);
        if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "upload hub layout");
    }
    if ((e = cudaGetLastError())) return cuda_error(ctx, e, "build buckets");
    return BISIM_OK;
}

}  // namespace bisim
