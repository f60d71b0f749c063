// bisim_refine_round_noalloc: one refinement round that allocates nothing.
//
// Some callers cannot allocate device memory at all: code running as a plugin
// inside another runtime that owns the whole device heap (a database engine's
// user-defined function, a custom operator of an inference server), or a
// latency-critical service loop that reserves every buffer up front because an
// allocation call may synchronise the device or fail under fragmentation. They
// pass their inputs and outputs; this entry point keeps all of its scratch in
// one fixed array compiled into the library (sized by kNoAlloc* below), which
// every GPU that loads the library holds until the process exits.
//
// The round itself is the same code as bisim_iterate's: the host-side round
// driver runs on a context that lives on the stack and whose buffers all point
// into the fixed array.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "prof.cuh"

namespace bisim {

namespace {

constexpr int64_t kNoAllocMaxVertices = 65536;
constexpr int64_t kNoAllocMaxEdges = 1 << 20;
constexpr int64_t kNoAllocMaxDegree = kMidMaxN;
constexpr int64_t kNoAllocSlots = 2 * kNoAllocMaxVertices;   // >= 2n, a power of two

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffTable = 0;
constexpr size_t kOffSkey = kOffTable + align256(sizeof(Slot) * kNoAllocSlots);
constexpr size_t kOffSlot = kOffSkey + align256(sizeof(unsigned long long) * kNoAllocMaxEdges);
constexpr size_t kOffCnt = kOffSlot + align256(sizeof(uint32_t) * kNoAllocMaxVertices);
constexpr size_t kOffList = kOffCnt + align256(sizeof(int32_t) * kNoAllocMaxVertices);
constexpr size_t kOffU0 = kOffList + align256(sizeof(int32_t) * kNoAllocMaxVertices);
constexpr size_t kOffU1 = kOffU0 + align256(sizeof(int32_t) * kNoAllocMaxVertices);
constexpr size_t kOffDefer = kOffU1 + align256(sizeof(int32_t) * kNoAllocMaxVertices);
constexpr size_t kOffState = kOffDefer + align256(sizeof(int32_t) * kNoAllocMaxVertices);
constexpr size_t kNoAllocBytes = kOffState + align256(sizeof(DevState));   // about 10.5 MB

// The fixed scratch. In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Checks the CSR and finds the largest out-degree; fills the identity vertex list.
__global__ void k_noalloc_prepare(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int32_t n,
                                  int64_t m, int32_t* __restrict__ list, DevState* st) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int64_t v = t0; v <= n; v += stride) {
        const int64_t a = rp[v];
        bool ok = a >= 0 && a <= m && (v != 0 || a == 0) && (v != n || a == m);
        if (v < n) {
            const int64_t b = rp[v + 1];
            ok = ok && b >= a;
            if (ok) atomicMax(&st->aux, static_cast<unsigned long long>(b - a));
            list[v] = static_cast<int32_t>(v);
        }
        if (!ok) atomicOr(&st->error, kErrBadInput);
    }
    for (int64_t e = t0; e < m; e += stride) {
        const int32_t d = col[e];
        if (d < 0 || d >= n) atomicOr(&st->error, kErrBadInput);
    }
}

std::mutex g_setup_mu;
unsigned char* g_scratch_addr[64] = {};

// Device address of the scratch array for the current device, looked up once
// per device.
cudaError_t scratch_address(int device, unsigned char** out) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (g_scratch_addr[device] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

// Whether the kernels of `device` may read or write `p` in place: managed
// memory, or device memory of that same device (memory of another GPU would
// need a peer mapping, which this call does not assume).
bool on_device(const void* p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

int mid_class_for(int64_t maxdeg) {
    int lg = 6;
    while ((int64_t{1} << lg) < maxdeg) ++lg;
    return lg - 6;   // N = 64 << class
}

}  // namespace

}  // namespace bisim

using namespace bisim;

extern "C" bisim_status bisim_refine_round_noalloc(int32_t n_vertices, int64_t n_edges, const int64_t* row_ptr,
                                                   const int32_t* col, const int32_t* edge_label,
                                                   const int32_t* block_in, int32_t* block_out,
                                                   int64_t* out_num_blocks, void* stream) {
    const int32_t n = n_vertices;
    const int64_t m = n_edges;
    if (n < 0 || m < 0) return set_error(nullptr, BISIM_EINVAL, "negative vertex or edge count");
    if (n > kNoAllocMaxVertices || m > kNoAllocMaxEdges)
        return set_error(nullptr, BISIM_EINVAL,
                         "graph exceeds the allocation-free limits (65536 vertices, 1048576 edges)");
    if (n == 0) {
        if (out_num_blocks) *out_num_blocks = 0;
        return BISIM_OK;
    }
    if (row_ptr == nullptr || block_in == nullptr || block_out == nullptr ||
        (m > 0 && (col == nullptr || edge_label == nullptr)))
        return set_error(nullptr, BISIM_EINVAL, "a required array is NULL");
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e) return cuda_error(nullptr, e, "cudaGetDevice");
    if (!on_device(row_ptr, device) || !on_device(block_in, device) || !on_device(block_out, device) ||
        (m > 0 && (!on_device(col, device) || !on_device(edge_label, device))))
        return set_error(nullptr, BISIM_EINVAL,
                         "the allocation-free round needs arrays in the current device's memory");
    if (block_in == block_out) return set_error(nullptr, BISIM_EINVAL, "block_in and block_out must differ");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* base = nullptr;
    if ((e = scratch_address(device, &base))) return cuda_error(nullptr, e, "cudaGetSymbolAddress(scratch)");

    // Every call starts from a blank table and status word: the array keeps
    // whatever the previous call left in it.
    uint64_t nslots = 1024;
    while (nslots < 2ull * static_cast<uint64_t>(n)) nslots <<= 1;
    DevState host_state;
    std::memset(&host_state, 0, sizeof(host_state));
    DevState* dstate = reinterpret_cast<DevState*>(base + kOffState);
    int32_t* list = reinterpret_cast<int32_t*>(base + kOffList);
    cudaMemsetAsync(base + kOffTable, 0, sizeof(Slot) * nslots, s);
    cudaMemsetAsync(dstate, 0, sizeof(DevState), s);
    {
        BISIM_SITE(site, "noalloc_prepare");
        Launch L(site, s, n, m, 8.0 * (n + 1) + 4.0 * m);
        const int64_t work = std::max<int64_t>(m, n + 1);
        k_noalloc_prepare<<<static_cast<unsigned>(std::min<int64_t>((work + 255) / 256, 4096)), 256, 0, s>>>(
            row_ptr, col, n, m, list, dstate);
    }
    // a launch that failed would leave the status word blank (largest degree 0)
    if ((e = cudaGetLastError())) return cuda_error(nullptr, e, "check CSR");
    cudaMemcpyAsync(&host_state, dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) return cuda_error(nullptr, e, "check CSR");
    if (host_state.error & kErrBadInput)
        return set_error(nullptr, BISIM_EINVAL, "malformed CSR: row_ptr not a prefix sum of [0, m] or a target out of range");
    const int64_t maxdeg = static_cast<int64_t>(host_state.aux);
    if (maxdeg > kNoAllocMaxDegree)
        return set_error(nullptr, BISIM_EINVAL, "an out-degree exceeds the allocation-free limit of 8192");

    // A context on the stack whose every buffer lies in the fixed array: all
    // vertices go through one degree class sized for the largest out-degree
    // (a warp per vertex up to 256 edges, a CTA per vertex above).
    bisim_ctx tc;
    tc.n = n;
    tc.m = m;
    bisim_default_options(&tc.opt);
    tc.opt.small_max_degree = 0;
    tc.opt.mid_max_degree = static_cast<int32_t>(kNoAllocMaxDegree);
    tc.device = device;
    tc.row_ptr = const_cast<int64_t*>(row_ptr);
    tc.col = const_cast<int32_t*>(col);
    tc.elab = const_cast<int32_t*>(edge_label);
    tc.P[0] = const_cast<int32_t*>(block_in);   // read only
    tc.P[1] = block_out;
    tc.cur = 0;
    tc.cnt = reinterpret_cast<int32_t*>(base + kOffCnt);
    tc.skey = reinterpret_cast<unsigned long long*>(base + kOffSkey);
    tc.slot = reinterpret_cast<uint32_t*>(base + kOffSlot);
    tc.table = reinterpret_cast<Slot*>(base + kOffTable);
    tc.nslots = nslots;
    tc.epoch32 = 0;
    tc.ulist[0] = reinterpret_cast<int32_t*>(base + kOffU0);
    tc.ulist[1] = reinterpret_cast<int32_t*>(base + kOffU1);
    tc.dlist = reinterpret_cast<int32_t*>(base + kOffDefer);
    tc.dstate = dstate;
    tc.hstate = &host_state;
    tc.class_list = list;
    const int cls = kSmallClasses + mid_class_for(maxdeg);
    for (int c = 0; c <= kNumClasses; ++c) tc.class_begin[c] = c <= cls ? 0 : n;
    tc.class_edges[cls] = m;
    int64_t blocks = 0;
    bisim_status st = refine_round(&tc, s, &blocks);
    if (st != BISIM_OK) return set_error(nullptr, st, tc.err);
    if (out_num_blocks) *out_num_blocks = blocks;
    return BISIM_OK;
}
