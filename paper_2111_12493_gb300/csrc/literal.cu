// Algorithm 4 taken literally (Section 3.3.1), as a diagnostic next to the
// exact refinement of the definition (Section 2.5).
//
// Algorithm 4 keeps two identifiers per vertex. id_s is refined like the
// definition for rounds 1 .. k-1: the own value and the set of
// (edge label, id_s of the neighbour). id_o carries no own value; its first
// round takes (edge label, id_o of the neighbour) and its later rounds only the
// neighbours' id_o. The final round k combines the own id_s with the set of the
// neighbours' id_o, without edge labels. For k = 1 the single round takes the
// own id_s and the set of (edge label, id_o of the neighbour). Both start from
// the label partition. With exact identifiers (no hash collisions) the result
// is a partition that the definition's P_k refines; where it is coarser, the
// literal algorithm merges classes the definition separates.
//
// A vertex without out-edges receives no message and keeps both identifiers
// (the worked example of Section 3.3.1 states this for v3 and v4); for id_s
// that is the same partition as hashing its own value with an empty set, for
// id_o it keeps the sinks apart by their previous id_o.
//
// Every step is one ordinary refinement round: the own term and the
// neighbour term come from different labellings by way of an auxiliary graph
// on 2n vertices, where vertex v keeps its out-edges but points them at w + n,
// and vertex w + n (no out-edges) carries the neighbour labelling shifted by n.
// The auxiliary copies never share a class with an original vertex, and the
// originals' canonical ids (smallest member) are unchanged by them. Each round
// runs through summarize_init_coo / bisim_iterate(k = 1) / get_partition.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "prof.cuh"

namespace bisim {

namespace {

unsigned grid_for(int64_t n, int threads) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 32)));
}

// Auxiliary graph: edges (u, w + n, keep_labels ? l : 0); labels own[v] for
// v < n, nb[v] + n for the copies (dead vertices keep -1); alive twice.
__global__ void k_aux_edges(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                            const int32_t* __restrict__ lab, int64_t m, int32_t n, bool keep_labels,
                            int32_t* __restrict__ as, int32_t* __restrict__ ad, int32_t* __restrict__ al) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += stride) {
        as[e] = src[e];
        ad[e] = dst[e] + n;
        al[e] = keep_labels ? lab[e] : 0;
    }
}

// Labels of the auxiliary graph. own == null (an id_o round): every vertex
// with out-edges gets 0, a vertex without any keeps its previous id_o (nb),
// stored as -2 - nb so that it meets neither 0, nor a copy (>= n), nor -1.
__global__ void k_aux_vertices(const int32_t* __restrict__ own, const int32_t* __restrict__ nb,
                               const int64_t* __restrict__ rp, const uint8_t* __restrict__ alive, int32_t n,
                               int32_t* __restrict__ vl, uint8_t* __restrict__ aalive) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += stride) {
        vl[v] = own ? own[v] : (rp[v + 1] == rp[v] ? -2 - nb[v] : 0);
        vl[v + n] = nb[v] < 0 ? -1 : nb[v] + n;
        const uint8_t a = alive ? alive[v] : 1;
        aalive[v] = a;
        aalive[v + n] = a;
    }
}

struct Lit {
    bisim_ctx* ctx;
    cudaStream_t s;
    int32_t n;
    int64_t m;
    const int32_t *src, *dst, *lab;
    // auxiliary scratch
    int32_t *as, *ad, *al, *avl, *apart;
    uint8_t* aalive;
};

// One refinement round of the labelling `own` on the context's graph (the
// ordinary round of the definition); result into out[n].
bisim_status round_plain(Lit& L, const int32_t* own, int32_t* out) {
    bisim_ctx* c = nullptr;
    bisim_options o;
    bisim_default_options(&o);
    o.hash_bits = L.ctx->opt.hash_bits;
    bisim_status st = summarize_init_coo(&c, L.n, L.m, L.src, L.dst, L.lab, own, L.ctx->alive, &o, L.s);
    if (st != BISIM_OK) return set_error(L.ctx, st, bisim_last_error(nullptr));
    int32_t r = 0;
    int64_t b = 0;
    if ((st = bisim_iterate(c, 1, 0, &r, &b, L.s)) == BISIM_OK) st = get_partition(c, out, L.s);
    if (st != BISIM_OK) set_error(L.ctx, st, bisim_last_error(c));
    summarize_destroy(c);
    return st;
}

// A round whose own term is `own` (null: an id_o round, see k_aux_vertices)
// and whose neighbour term is `nb`, with or without the edge labels; result
// into out[n].
bisim_status round_split(Lit& L, const int32_t* own, const int32_t* nb, bool labels, int32_t* out) {
    const int32_t n = L.n;
    BISIM_SITE(site, "literal_aux");
    {
        Launch K(site, L.s, 2 * n, L.m, 12.0 * L.m + 16.0 * n);
        if (L.m > 0)
            k_aux_edges<<<grid_for(L.m, 256), 256, 0, L.s>>>(L.src, L.dst, L.lab, L.m, n, labels, L.as, L.ad, L.al);
        k_aux_vertices<<<grid_for(n, 256), 256, 0, L.s>>>(own, nb, L.ctx->row_ptr, L.ctx->alive, n, L.avl, L.aalive);
    }
    bisim_ctx* c = nullptr;
    bisim_options o;
    bisim_default_options(&o);
    o.hash_bits = L.ctx->opt.hash_bits;
    bisim_status st = summarize_init_coo(&c, 2 * n, L.m, L.as, L.ad, L.al, L.avl, L.aalive, &o, L.s);
    if (st != BISIM_OK) return set_error(L.ctx, st, bisim_last_error(nullptr));
    int32_t r = 0;
    int64_t b = 0;
    if ((st = bisim_iterate(c, 1, 0, &r, &b, L.s)) == BISIM_OK) st = get_partition(c, L.apart, L.s);
    if (st != BISIM_OK) set_error(L.ctx, st, bisim_last_error(c));
    summarize_destroy(c);
    if (st != BISIM_OK) return st;
    cudaMemcpyAsync(out, L.apart, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, L.s);
    return BISIM_OK;
}

}  // namespace

}  // namespace bisim

using namespace bisim;

extern "C" bisim_status bisim_literal_alg4(bisim_ctx* ctx, int32_t k, int32_t* block, int64_t* out_num_blocks,
                                           void* stream) {
    if (ctx == nullptr) return set_error(nullptr, BISIM_EINVAL, "ctx is NULL");
    ctx->last_stream = stream;
    if (k < 0) return set_error(ctx, BISIM_EINVAL, "k must be >= 0");
    if (ctx->gid != nullptr) return set_error(ctx, BISIM_ESTATE, "batched contexts have no literal mode");
    if (ctx->n > (1 << 30)) return set_error(ctx, BISIM_EINVAL, "the literal mode needs 2n vertices to fit int32");
    if (block == nullptr && ctx->n > 0) return set_error(ctx, BISIM_EINVAL, "output is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    bisim_status st;
    if ((st = refresh_after_edit(ctx, s)) != BISIM_OK || (st = ensure_vertex_csr(ctx, s)) != BISIM_OK) return st;
    const int32_t n = ctx->n;
    const int64_t m = ctx->m;
    if (n == 0) {
        if (out_num_blocks) *out_num_blocks = 0;
        return BISIM_OK;
    }
    const size_t nn = static_cast<size_t>(n), mm = static_cast<size_t>(std::max<int64_t>(m, 1));
    // scratch: the edge sources, the auxiliary graph, five labellings of n and two of 2n vertices
    std::vector<void*> bufs;
    auto get = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) return nullptr;
        bufs.push_back(p);
        return p;
    };
    Lit L{ctx, s, n, m, nullptr, ctx->col, ctx->elab, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int32_t* src = static_cast<int32_t*>(get(4 * mm));
    L.as = static_cast<int32_t*>(get(4 * mm));
    L.ad = static_cast<int32_t*>(get(4 * mm));
    L.al = static_cast<int32_t*>(get(4 * mm));
    L.avl = static_cast<int32_t*>(get(8 * nn));
    L.apart = static_cast<int32_t*>(get(8 * nn));
    L.aalive = static_cast<uint8_t*>(get(2 * nn));
    int32_t* ids = static_cast<int32_t*>(get(4 * nn));
    int32_t* ido = static_cast<int32_t*>(get(4 * nn));
    int32_t* t1 = static_cast<int32_t*>(get(4 * nn));
    int32_t* t2 = static_cast<int32_t*>(get(4 * nn));
    auto release = [&]() {
        for (void* p : bufs) cudaFreeAsync(p, s);
        bufs.clear();
    };
    for (void* p : bufs)
        if (p == nullptr) {
            release();
            cudaGetLastError();
            return set_error(ctx, BISIM_ENOMEM, "alloc literal-mode scratch");
        }
    if (bufs.size() != 11) {
        release();
        cudaGetLastError();
        return set_error(ctx, BISIM_ENOMEM, "alloc literal-mode scratch");
    }
    L.src = src;
    if (m > 0 && (st = csr_sources(ctx, ctx->row_ptr, n, m, src, s)) != BISIM_OK) {
        release();
        return st;
    }
    // initialization: id_s = id_o = the label partition
    cudaMemcpyAsync(ids, ctx->P0, sizeof(int32_t) * nn, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(ido, ctx->P0, sizeof(int32_t) * nn, cudaMemcpyDeviceToDevice, s);
    st = BISIM_OK;
    if (k == 1) {
        // the single round: own id_s and the set of (label, id_o of the neighbour)
        st = round_split(L, ids, ido, true, t1);
        if (st == BISIM_OK) std::swap(ids, t1);
    } else if (k >= 2) {
        for (int32_t i = 1; i <= k - 1 && st == BISIM_OK; ++i) {
            // id_s: own id_s and (label, id_s of the neighbour); id_o: no own term,
            // (label, id_o) in the first round, then the neighbours' id_o alone
            st = round_plain(L, ids, t1);
            if (st == BISIM_OK) st = round_split(L, nullptr, ido, i == 1, t2);
            if (st == BISIM_OK) {
                std::swap(ids, t1);
                std::swap(ido, t2);
            }
        }
        // final round: own id_s and the set of the neighbours' id_o, no labels
        if (st == BISIM_OK) st = round_split(L, ids, ido, false, t1);
        if (st == BISIM_OK) std::swap(ids, t1);
    }
    if (st == BISIM_OK && (e = cudaMemcpyAsync(block, ids, sizeof(int32_t) * nn, cudaMemcpyDefault, s))) {
        release();
        return cuda_error(ctx, e, "copy literal-mode partition");
    }
    int64_t blocks = 0;
    if (st == BISIM_OK && out_num_blocks) {
        // blocks = vertices that are their own block id
        std::vector<int32_t> h(nn);
        if ((e = cudaMemcpyAsync(h.data(), ids, sizeof(int32_t) * nn, cudaMemcpyDeviceToHost, s)) ||
            (e = cudaStreamSynchronize(s))) {
            release();
            return cuda_error(ctx, e, "literal mode");
        }
        for (int32_t v = 0; v < n; ++v) blocks += h[v] == v ? 1 : 0;
        *out_num_blocks = blocks;
    }
    release();
    if (st != BISIM_OK) return st;
    if ((e = cudaStreamSynchronize(s))) return cuda_error(ctx, e, "literal mode");
    return BISIM_OK;
}
