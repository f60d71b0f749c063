// Direction and label parameterizations (Section 2.4.2 and Section 2.5):
// forward bisimulation compares the out-edges of two vertices, backward
// bisimulation their in-edges, and the forward-backward variant both; a label
// filter restricts the edges taken into account to a set of labels.
//
// The refinement kernels always compare out-edges of the graph they are given,
// so each variant becomes an edge list that the unchanged path refines:
//   forward     the edges as given
//   backward    every edge (u, w, l) reversed to (w, u, l)
//   both        every edge twice: (u, w, 2l) for the out-edge of u and
//               (w, u, 2l + 1) for the in-edge of w, so a pair's label keeps
//               its direction and no out-pair can equal an in-pair (labels
//               must lie in [-2^30, 2^30) for this to be injective)
//   filter      edges whose label is not listed are left out
// Update batches go through the same mapping (an edge operation becomes one
// or two operations on the internal edge list, in order), and the summary
// graph reports edges in the caller's direction and labels.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "prof.cuh"

namespace bisim {

namespace {

constexpr int32_t kBothLabelMin = -(1 << 30);
constexpr int32_t kBothLabelMax = (1 << 30) - 1;

unsigned grid_for(int64_t n, int threads) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 32)));
}

__device__ __forceinline__ bool listed(const int32_t* __restrict__ f, int32_t nf, int32_t l) {
    if (nf == 0) return true;
    int32_t lo = 0, hi = nf - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (f[mid] < l) lo = mid + 1; else hi = mid;
    }
    return f[lo] == l;
}

// Internal edges per input edge (0, 1 or 2); cnt[m] = 0 closes the scan.
__global__ void k_view_count(const int32_t* __restrict__ lab, int64_t m, const int32_t* __restrict__ filt, int32_t nf,
                             int32_t dir, int64_t* __restrict__ cnt, unsigned* err) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e <= m; e += stride) {
        if (e == m) {
            cnt[e] = 0;
            continue;
        }
        const int32_t l = lab[e];
        const bool keep = listed(filt, nf, l);
        if (keep && dir == BISIM_DIR_BOTH && (l < kBothLabelMin || l > kBothLabelMax)) atomicOr(err, kErrBadInput);
        cnt[e] = keep ? (dir == BISIM_DIR_BOTH ? 2 : 1) : 0;
    }
}

__global__ void k_view_emit(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                            const int32_t* __restrict__ lab, int64_t m, const int64_t* __restrict__ pos, int32_t dir,
                            int32_t* __restrict__ os, int32_t* __restrict__ od, int32_t* __restrict__ ol) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int64_t p = pos[e];
        if (pos[e + 1] == p) continue;
        const int32_t u = src[e], w = dst[e], l = lab[e];
        if (dir == BISIM_DIR_FORWARD) {
            os[p] = u; od[p] = w; ol[p] = l;
        } else if (dir == BISIM_DIR_BACKWARD) {
            os[p] = w; od[p] = u; ol[p] = l;
        } else {
            os[p] = u; od[p] = w; ol[p] = 2 * l;
            os[p + 1] = w; od[p + 1] = u; ol[p + 1] = 2 * l + 1;
        }
    }
}

__global__ void k_view_offsets(const int64_t* __restrict__ pos, const int64_t* __restrict__ eoff, int32_t G,
                               int64_t* __restrict__ out) {
    const int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g <= G) out[g] = pos[eoff[g]];
}

// Internal operations per operation: edge operations as edges above, vertex
// operations (and unknown kinds, which the batch check rejects) once.
__global__ void k_ops_count(const bisim_op* __restrict__ ops, int64_t n, const int32_t* __restrict__ filt, int32_t nf,
                            int32_t dir, int64_t* __restrict__ cnt, unsigned* err) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i <= n; i += stride) {
        if (i == n) {
            cnt[i] = 0;
            continue;
        }
        const bisim_op o = ops[i];
        int64_t c = 1;
        if (o.kind == BISIM_OP_EDGE_ADD || o.kind == BISIM_OP_EDGE_DEL) {
            const bool keep = listed(filt, nf, o.label);
            if (keep && dir == BISIM_DIR_BOTH && (o.label < kBothLabelMin || o.label > kBothLabelMax))
                atomicOr(err, kErrBadInput);
            c = keep ? (dir == BISIM_DIR_BOTH ? 2 : 1) : 0;
        }
        cnt[i] = c;
    }
}

__global__ void k_ops_emit(const bisim_op* __restrict__ ops, int64_t n, const int64_t* __restrict__ pos, int32_t dir,
                           bisim_op* __restrict__ out) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t p = pos[i];
        if (pos[i + 1] == p) continue;
        bisim_op o = ops[i];
        if (o.kind != BISIM_OP_EDGE_ADD && o.kind != BISIM_OP_EDGE_DEL) {
            out[p] = o;
        } else if (dir == BISIM_DIR_FORWARD) {
            out[p] = o;
        } else if (dir == BISIM_DIR_BACKWARD) {
            out[p] = bisim_op{o.kind, o.dst, o.src, o.label};
        } else {
            out[p] = bisim_op{o.kind, o.src, o.dst, 2 * o.label};
            out[p + 1] = bisim_op{o.kind, o.dst, o.src, 2 * o.label + 1};
        }
    }
}

// One warp per vertex writes the vertex into its row's entries; rows outside
// [0, m] or running backwards only raise the error flag.
__global__ void k_csr_sources(const int64_t* __restrict__ rp, int32_t n, int64_t m, int32_t* __restrict__ src,
                              unsigned* err) {
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    const unsigned lane = threadIdx.x & 31u;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); v <= n; v += warps) {
        const int64_t a = rp[v];
        if (v == n) {
            if (lane == 0 && a != m) atomicOr(err, kErrBadInput);
            continue;
        }
        const int64_t b = rp[v + 1];
        if (a < 0 || b < a || b > m || (v == 0 && a != 0)) {
            if (lane == 0) atomicOr(err, kErrBadInput);
            continue;
        }
        for (int64_t e = a + lane; e < b; e += 32) src[e] = static_cast<int32_t>(v);
    }
}

}  // namespace

bisim_status csr_sources(bisim_ctx* ctx, const int64_t* row_ptr, int32_t n, int64_t m, int32_t* src, cudaStream_t s) {
    cudaMemsetAsync(&ctx->dstate->error, 0, sizeof(unsigned), s);
    BISIM_SITE(site, "csr_sources");
    {
        Launch L(site, s, n, m, 8.0 * n + 4.0 * m);
        k_csr_sources<<<grid_for(static_cast<int64_t>(n + 1) * 32, 256), 256, 0, s>>>(row_ptr, n, m, src,
                                                                                     &ctx->dstate->error);
    }
    unsigned err = 0;
    cudaError_t e;
    cudaMemcpyAsync(&err, &ctx->dstate->error, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "CSR sources");
    if (err & kErrBadInput) return set_error(ctx, BISIM_EINVAL, "row_ptr is not a prefix sum of [0, m]");
    return BISIM_OK;
}

bool edge_view_identity(const bisim_ctx* ctx) {
    return ctx->opt.direction == BISIM_DIR_FORWARD && ctx->nfilter == 0;
}

bisim_status edge_view_setup(bisim_ctx* ctx, const bisim_options* opt, cudaStream_t s) {
    ctx->opt.label_filter = nullptr;                // caller memory: never kept
    if (opt == nullptr || opt->n_label_filter <= 0) return BISIM_OK;
    if (opt->label_filter == nullptr) return set_error(ctx, BISIM_EINVAL, "label_filter is NULL");
    std::vector<int32_t> f(static_cast<size_t>(opt->n_label_filter));
    cudaError_t e;
    if ((e = cudaMemcpyAsync(f.data(), opt->label_filter, sizeof(int32_t) * f.size(), cudaMemcpyDefault, s)) ||
        (e = cudaStreamSynchronize(s)))
        return cuda_error(ctx, e, "read label filter");
    std::sort(f.begin(), f.end());
    f.erase(std::unique(f.begin(), f.end()), f.end());
    if ((e = ctx_alloc(ctx, reinterpret_cast<void**>(&ctx->dfilter), sizeof(int32_t) * f.size(), s)))
        return cuda_error(ctx, e, "alloc label filter");
    ctx->nfilter = static_cast<int32_t>(f.size());
    if ((e = cudaMemcpyAsync(ctx->dfilter, f.data(), sizeof(int32_t) * f.size(), cudaMemcpyHostToDevice, s)) ||
        (e = cudaStreamSynchronize(s)))
        return cuda_error(ctx, e, "upload label filter");
    return BISIM_OK;
}

bisim_status edge_view_coo(bisim_ctx* ctx, const int32_t* src, const int32_t* dst, const int32_t* lab, int64_t m,
                           const int64_t* eoff, int32_t G, cudaStream_t s, EdgeView* out) {
    *out = EdgeView{};
    cudaError_t e;
    const size_t scan_words = scan_temp_words(m + 1);
    int64_t* pos = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&pos), sizeof(int64_t) * (2 * (m + 1) + scan_words), s)))
        return cuda_error(ctx, e, "alloc edge view");
    int64_t* cnt = pos + (m + 1);
    int64_t* tmp = cnt + (m + 1);
    const int32_t dir = ctx->opt.direction;
    cudaMemsetAsync(&ctx->dstate->error, 0, sizeof(unsigned), s);
    BISIM_SITE(site, "edge_view");
    {
        Launch L(site, s, 0, m, 24.0 * m);
        k_view_count<<<grid_for(m + 1, 256), 256, 0, s>>>(lab, m, ctx->dfilter, ctx->nfilter, dir, cnt,
                                                          &ctx->dstate->error);
    }
    exclusive_scan_i64(cnt, pos, m + 1, tmp, s);
    int64_t total = 0;
    unsigned err = 0;
    cudaMemcpyAsync(&total, pos + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&err, &ctx->dstate->error, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) {
        cudaFreeAsync(pos, s);
        return cuda_error(ctx, e, "count edge view");
    }
    if (err & kErrBadInput) {
        cudaFreeAsync(pos, s);
        return set_error(ctx, BISIM_EINVAL, "the forward-backward direction needs edge labels in [-2^30, 2^30)");
    }
    const size_t eb = sizeof(int32_t) * static_cast<size_t>(std::max<int64_t>(total, 1));
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&out->src), eb, s)) ||
        (e = cudaMallocAsync(reinterpret_cast<void**>(&out->dst), eb, s)) ||
        (e = cudaMallocAsync(reinterpret_cast<void**>(&out->lab), eb, s)) ||
        (eoff && (e = cudaMallocAsync(reinterpret_cast<void**>(&out->eoff), sizeof(int64_t) * (G + 1), s)))) {
        cudaFreeAsync(pos, s);
        edge_view_free(out, s);
        return cuda_error(ctx, e, "alloc edge view");
    }
    {
        Launch L(site, s, 0, m, 24.0 * m + 12.0 * total);
        k_view_emit<<<grid_for(m, 256), 256, 0, s>>>(src, dst, lab, m, pos, dir, out->src, out->dst, out->lab);
        if (eoff) k_view_offsets<<<(G + 256) / 256, 256, 0, s>>>(pos, eoff, G, out->eoff);
    }
    out->m = total;
    cudaFreeAsync(pos, s);
    if ((e = cudaGetLastError())) return cuda_error(ctx, e, "edge view");
    return BISIM_OK;
}

void edge_view_free(EdgeView* v, cudaStream_t s) {
    if (v->src) cudaFreeAsync(v->src, s);
    if (v->dst) cudaFreeAsync(v->dst, s);
    if (v->lab) cudaFreeAsync(v->lab, s);
    if (v->eoff) cudaFreeAsync(v->eoff, s);
    *v = EdgeView{};
}

bisim_status edge_view_ops(bisim_ctx* ctx, const bisim_op* ops, int64_t n, cudaStream_t s, bisim_op** out,
                           int64_t* out_n) {
    *out = nullptr;
    *out_n = 0;
    cudaError_t e;
    const size_t scan_words = scan_temp_words(n + 1);
    int64_t* pos = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&pos), sizeof(int64_t) * (2 * (n + 1) + scan_words), s)))
        return cuda_error(ctx, e, "alloc op view");
    int64_t* cnt = pos + (n + 1);
    int64_t* tmp = cnt + (n + 1);
    const int32_t dir = ctx->opt.direction;
    cudaMemsetAsync(&ctx->dstate->error, 0, sizeof(unsigned), s);
    k_ops_count<<<grid_for(n + 1, 256), 256, 0, s>>>(ops, n, ctx->dfilter, ctx->nfilter, dir, cnt, &ctx->dstate->error);
    exclusive_scan_i64(cnt, pos, n + 1, tmp, s);
    int64_t total = 0;
    unsigned err = 0;
    cudaMemcpyAsync(&total, pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&err, &ctx->dstate->error, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) {
        cudaFreeAsync(pos, s);
        return cuda_error(ctx, e, "count op view");
    }
    if (err & kErrBadInput) {
        cudaFreeAsync(pos, s);
        return set_error(ctx, BISIM_EINVAL, "the forward-backward direction needs edge labels in [-2^30, 2^30)");
    }
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(out), sizeof(bisim_op) * std::max<int64_t>(total, 1), s))) {
        cudaFreeAsync(pos, s);
        return cuda_error(ctx, e, "alloc op view");
    }
    k_ops_emit<<<grid_for(n, 256), 256, 0, s>>>(ops, n, pos, dir, *out);
    cudaFreeAsync(pos, s);
    if ((e = cudaGetLastError())) return cuda_error(ctx, e, "op view");
    *out_n = total;
    return BISIM_OK;
}

}  // namespace bisim
