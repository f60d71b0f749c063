// The summary graph of the current partition: its vertices' payload (the
// number of vertices each block summarizes) and its edges.
//
// Section 2.6 defines the graph summary SG: one vertex per equivalence class,
// and an edge labelled l from the class of u to the class of w for the edges
// (u, w) of the data graph with label l; parallel edges of one label between
// two classes collapse into one. Section 3.1 names counting the summarized
// vertices as the typical payload, merged by adding counts when vertex
// summaries merge. For the partition P held by a context:
//
//   size(b)  = |{ v : P[v] = b }|                          (b a block id)
//   E_vs     = { (P[u], l, P[w]) : (u, w, l) a live edge }  (a set)
//
// The edges are produced by three stable LSD radix sorts of the edges' triples
// (target block, then label, then source block), which leaves them in
// lexicographic order, and one pass that keeps the first of every run of
// equal triples.
#include <algorithm>
#include <cstddef>
#include <vector>

#include "common.cuh"
#include "prof.cuh"

namespace bisim {

namespace {

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

unsigned grid_for(int64_t n, int threads) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(cdiv(n, threads), 152 * 32)));
}

int bits_for(int64_t n) {
    int b = 0;
    while ((int64_t{1} << b) < n) ++b;
    return std::max(b, 1);
}

constexpr uint32_t kLabelFlip = 0x80000000u;   // signed labels sort in signed order as unsigned keys

__global__ void k_block_sizes(const int32_t* __restrict__ P, int32_t n, int32_t* __restrict__ sizes) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t b = P[v];
        if (b >= 0) atomicAdd(&sizes[b], 1);
    }
}

// The last vertex v with rp[v] <= e (rp non-decreasing, rp[0] = 0 <= e < rp[n]),
// searched in [lo, hi].
__device__ __forceinline__ int32_t row_of(const int64_t* __restrict__ rp, int64_t e, int32_t lo, int32_t hi) {
    while (lo < hi) {
        const int32_t mid = lo + (hi - lo + 1) / 2;
        if (rp[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Pass A keys: every edge's target block (key) with (source block, flipped
// label) as the value. Edges with a dead endpoint get the source block n, so
// that they sort after every live triple. Each CTA takes a tile of edges and
// narrows the search for their source rows to the rows the tile spans.
constexpr int kKeyTile = 2048;
// The context's own edges map back to the caller's (direction.cu): backward
// contexts hold every edge reversed; forward-backward contexts hold (u, w, 2l)
// and the in-edge copy (w, u, 2l + 1), which is left out here.
__global__ void __launch_bounds__(256) k_summary_keys(const int64_t* __restrict__ rp, int32_t n,
                                                      const int32_t* __restrict__ col,
                                                      const int32_t* __restrict__ elab, int64_t m,
                                                      const int32_t* __restrict__ P, int32_t dir,
                                                      uint32_t* __restrict__ key, uint64_t* __restrict__ val) {
    __shared__ int32_t span[2];
    const int64_t tiles = cdiv(m, kKeyTile);
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t e0 = t * kKeyTile;
        const int64_t e1 = e0 + kKeyTile < m ? e0 + kKeyTile : m;
        if (threadIdx.x < 2) span[threadIdx.x] = row_of(rp, threadIdx.x == 0 ? e0 : e1 - 1, 0, n - 1);
        __syncthreads();
        const int32_t lo = span[0], hi = span[1];
        for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const int32_t u = row_of(rp, e, lo, hi);
            int32_t sb = P[u], tb = P[col[e]], l = elab[e];
            bool live = sb >= 0 && tb >= 0;
            if (dir == BISIM_DIR_BACKWARD) {
                const int32_t t = sb;
                sb = tb;
                tb = t;
            } else if (dir == BISIM_DIR_BOTH) {
                live = live && (l & 1) == 0;
                l >>= 1;                                   // arithmetic: 2l -> l for negative l too
            }
            key[e] = live ? static_cast<uint32_t>(tb) : 0u;
            val[e] = (static_cast<uint64_t>(live ? static_cast<uint32_t>(sb) : static_cast<uint32_t>(n)) << 32) |
                     (static_cast<uint32_t>(l) ^ kLabelFlip);
        }
        __syncthreads();
    }
}

// After pass A (key = target block, value = source << 32 | label): key = label,
// value = source << 32 | target.
__global__ void k_summary_to_label(const uint32_t* __restrict__ ki, const uint64_t* __restrict__ vi, int64_t m,
                                   uint32_t* __restrict__ ko, uint64_t* __restrict__ vo) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint64_t v = vi[e];
        ko[e] = static_cast<uint32_t>(v);
        vo[e] = (v & 0xffffffff00000000ull) | ki[e];
    }
}

// After pass B (key = label, value = source << 32 | target): key = source,
// value = label << 32 | target.
__global__ void k_summary_to_source(const uint32_t* __restrict__ ki, const uint64_t* __restrict__ vi, int64_t m,
                                    uint32_t* __restrict__ ko, uint64_t* __restrict__ vo) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint64_t v = vi[e];
        ko[e] = static_cast<uint32_t>(v >> 32);
        vo[e] = (static_cast<uint64_t>(ki[e]) << 32) | static_cast<uint32_t>(v);
    }
}

// Sorted triples (key = source, value = label << 32 | target): 1 for the first
// of every run of equal live triples.
__global__ void k_summary_heads(const uint32_t* __restrict__ k, const uint64_t* __restrict__ v, int64_t m,
                                int32_t n, int64_t* __restrict__ head) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e <= m; e += stride) {
        if (e == m) {
            head[e] = 0;
            continue;
        }
        const bool live = k[e] < static_cast<uint32_t>(n);
        head[e] = live && (e == 0 || k[e] != k[e - 1] || v[e] != v[e - 1]) ? 1 : 0;
    }
}

__global__ void k_summary_emit(const uint32_t* __restrict__ k, const uint64_t* __restrict__ v, int64_t m,
                               int32_t n, const int64_t* __restrict__ at, int32_t* __restrict__ os,
                               int32_t* __restrict__ ol, int32_t* __restrict__ ot) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += stride) {
        if (at[e + 1] == at[e]) continue;                    // not the head of a run
        const int64_t i = at[e];
        os[i] = static_cast<int32_t>(k[e]);
        ol[i] = static_cast<int32_t>(static_cast<uint32_t>(v[e] >> 32) ^ kLabelFlip);
        ot[i] = static_cast<int32_t>(static_cast<uint32_t>(v[e]));
    }
}

}  // namespace

}  // namespace bisim

using namespace bisim;

extern "C" {

bisim_status get_block_sizes(bisim_ctx* ctx, int32_t* sizes, void* stream) {
    if (ctx == nullptr) return set_error(nullptr, BISIM_EINVAL, "ctx is NULL");
    ctx->last_stream = stream;
    if (ctx->n == 0) return BISIM_OK;
    if (sizes == nullptr) return set_error(ctx, BISIM_EINVAL, "output is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    int32_t* d = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&d), sizeof(int32_t) * ctx->n, s)))
        return cuda_error(ctx, e, "alloc block sizes");
    cudaMemsetAsync(d, 0, sizeof(int32_t) * ctx->n, s);
    BISIM_SITE(site, "block_sizes");
    {
        Launch L(site, s, ctx->n, 0, 8.0 * ctx->n);
        k_block_sizes<<<grid_for(ctx->n, 256), 256, 0, s>>>(ctx->P[ctx->cur], ctx->n, d);
    }
    e = cudaMemcpyAsync(sizes, d, sizeof(int32_t) * ctx->n, cudaMemcpyDefault, s);
    cudaFreeAsync(d, s);
    if (e || (e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "block sizes");
    return BISIM_OK;
}

bisim_status get_summary_edges(bisim_ctx* ctx, int32_t* src_block, int32_t* label, int32_t* dst_block,
                               int64_t capacity, int64_t* out_count, void* stream) {
    if (ctx == nullptr) return set_error(nullptr, BISIM_EINVAL, "ctx is NULL");
    ctx->last_stream = stream;
    if (out_count == nullptr || capacity < 0) return set_error(ctx, BISIM_EINVAL, "invalid count or capacity");
    if (capacity > 0 && (src_block == nullptr || label == nullptr || dst_block == nullptr))
        return set_error(ctx, BISIM_EINVAL, "an output array is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    bisim_status st;
    *out_count = 0;
    if ((st = ensure_vertex_csr(ctx, s)) != BISIM_OK) return st;
    const int32_t n = ctx->n;
    const int64_t m = ctx->m;
    if (n == 0 || m == 0) return BISIM_OK;
    // scratch: keys and values twice (radix ping-pong), run heads and their offsets, the radix temp,
    // the compacted triples
    const size_t tmp_words = std::max(radix_temp_words(m), scan_temp_words(m + 1));
    // every piece starts on a 256-byte boundary: the allocation is the sum of the rounded sizes
    auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t mm = static_cast<size_t>(m);
    const size_t bytes = 2 * r256(sizeof(uint32_t) * mm) + 2 * r256(sizeof(uint64_t) * mm) +
                         2 * r256(sizeof(int64_t) * (mm + 1)) + r256(sizeof(int64_t) * tmp_words) +
                         3 * r256(sizeof(int32_t) * mm);
    char* base = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&base), bytes, s))) return cuda_error(ctx, e, "alloc summary scratch");
    char* cur = base;
    auto carve = [&](size_t b) { char* p = cur; cur += r256(b); return p; };
    uint32_t* k0 = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * m));
    uint32_t* k1 = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * m));
    uint64_t* v0 = reinterpret_cast<uint64_t*>(carve(sizeof(uint64_t) * m));
    uint64_t* v1 = reinterpret_cast<uint64_t*>(carve(sizeof(uint64_t) * m));
    int64_t* head = reinterpret_cast<int64_t*>(carve(sizeof(int64_t) * (m + 1)));
    int64_t* at = reinterpret_cast<int64_t*>(carve(sizeof(int64_t) * (m + 1)));
    int64_t* tmp = reinterpret_cast<int64_t*>(carve(sizeof(int64_t) * tmp_words));
    int32_t* os = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * m));
    int32_t* ol = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * m));
    int32_t* ot = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * m));
    const int32_t* P = ctx->P[ctx->cur];
    BISIM_SITE(site, "summary_edges");
    int64_t count = 0;
    {
        Launch L(site, s, n, m, 48.0 * m);
        k_summary_keys<<<grid_for(cdiv(m, kKeyTile) * 256, 256), 256, 0, s>>>(ctx->row_ptr, n, ctx->col, ctx->elab, m,
                                                                                P, ctx->opt.direction, k0, v0);
    }
    // pass A: by target block (stable), the result in (k0, v0) or (k1, v1)
    int w = radix_sort_pairs(k0, v0, k1, v1, m, bits_for(n), tmp, s, "summary_radix");
    uint32_t* ka = w ? k1 : k0;
    uint64_t* va = w ? v1 : v0;
    uint32_t* kb = w ? k0 : k1;
    uint64_t* vb = w ? v0 : v1;
    k_summary_to_label<<<grid_for(m, 256), 256, 0, s>>>(ka, va, m, kb, vb);
    // pass B: by label
    w = radix_sort_pairs(kb, vb, ka, va, m, 32, tmp, s, "summary_radix");
    uint32_t* kc = w ? ka : kb;
    uint64_t* vc = w ? va : vb;
    uint32_t* kd = w ? kb : ka;
    uint64_t* vd = w ? vb : va;
    k_summary_to_source<<<grid_for(m, 256), 256, 0, s>>>(kc, vc, m, kd, vd);
    // pass C: by source block (dead-endpoint edges carry n and sort last)
    w = radix_sort_pairs(kd, vd, kc, vc, m, bits_for(static_cast<int64_t>(n) + 1), tmp, s, "summary_radix");
    const uint32_t* kf = w ? kc : kd;
    const uint64_t* vf = w ? vc : vd;
    {
        Launch L(site, s, 0, m, 36.0 * m);
        k_summary_heads<<<grid_for(m + 1, 256), 256, 0, s>>>(kf, vf, m, n, head);
        exclusive_scan_i64(head, at, m + 1, tmp, s);
        k_summary_emit<<<grid_for(m, 256), 256, 0, s>>>(kf, vf, m, n, at, os, ol, ot);
    }
    cudaMemcpyAsync(&count, at + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) {
        cudaFreeAsync(base, s);
        return cuda_error(ctx, e, "summary edges");
    }
    if (cur - base != static_cast<ptrdiff_t>(bytes) || count < 0 || count > m) {
        cudaFreeAsync(base, s);
        return set_error(ctx, BISIM_ECUDA, "summary edges: inconsistent scratch layout or count");
    }
    const int64_t take = std::min(capacity, count);
    if (take > 0) {
        cudaMemcpyAsync(src_block, os, sizeof(int32_t) * take, cudaMemcpyDefault, s);
        cudaMemcpyAsync(label, ol, sizeof(int32_t) * take, cudaMemcpyDefault, s);
        cudaMemcpyAsync(dst_block, ot, sizeof(int32_t) * take, cudaMemcpyDefault, s);
    }
    cudaFreeAsync(base, s);
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "copy summary edges");
    *out_count = count;
    return BISIM_OK;
}

}  // extern "C"
