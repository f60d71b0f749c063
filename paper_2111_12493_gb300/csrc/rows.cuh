// Work over the entries of many rows whose lengths range from a few entries
// to a million (power-law degrees). Every row is a task; a producer files it
// in one of three tiers by length and each tier gets a matching share of the
// GPU:
//   warp tier  len <= kWarpTierMax   one warp per task
//   CTA tier   len <= kCtaTierMax    one CTA per task, its warps striding the row
//   grid tier  longer                the row's 32-entry chunks go round-robin to every warp
// The consumer is a persistent grid that reads the task counts on the device,
// so filing and consuming need no host round trip. The per-entry work is a
// functor called by whole warps (`in` is false past the row's end), so it may
// use warp collectives.
#pragma once

#include "common.cuh"

namespace bisim {

struct RowTask {
    int64_t off;      // first entry
    int32_t len;      // entries
    int32_t arg;      // the producer's tag (a vertex, a key slot, ...)
};

constexpr int32_t kWarpTierMax = 512;
constexpr int32_t kCtaTierMax = 16384;
constexpr int kTierThreads = 256;
constexpr int kTierGrid = 152 * 4;

struct TierLists {
    RowTask* t[3];
    unsigned* cnt;    // [3], on the device
};

__device__ __forceinline__ int tier_of(int32_t len) {
    return len <= kWarpTierMax ? 0 : len <= kCtaTierMax ? 1 : 2;
}

// Files `task` for every lane with `has` (and a non-empty row). All 32 lanes
// of the warp must call it together.
__device__ __forceinline__ void tier_push(const TierLists& L, bool has, const RowTask& task) {
    const unsigned lane = threadIdx.x & 31u;
    const int k = tier_of(task.len);
    const bool mine = has && task.len > 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const unsigned b = __ballot_sync(0xffffffffu, mine && k == q);
        if (b == 0u) continue;
        const int leader = __ffs(b) - 1;
        unsigned base = 0;
        if (static_cast<int>(lane) == leader) base = atomicAdd(&L.cnt[q], static_cast<unsigned>(__popc(b)));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (mine && k == q) L.t[q][base + __popc(b & ((1u << lane) - 1u))] = task;
    }
}

// One persistent grid runs the three tiers in turn: the warp tier's tasks over
// all warps, then the CTA tier's over all CTAs, then every grid-tier row over
// all warps together. Tasks are independent, so no grid-wide barrier is needed
// between the phases.
template <class F>
__global__ void __launch_bounds__(kTierThreads) k_tiers(const TierLists L, F f, bool grid_tier) {
    const int lane = static_cast<int>(threadIdx.x & 31u);
    const int warp = static_cast<int>(threadIdx.x >> 5);
    const unsigned warps = gridDim.x * (kTierThreads / 32);
    const unsigned gw = blockIdx.x * (kTierThreads / 32) + warp;
    const unsigned c0 = *reinterpret_cast<volatile unsigned*>(&L.cnt[0]);
    for (unsigned i = gw; i < c0; i += warps) {
        const RowTask t = L.t[0][i];
        for (int32_t j0 = 0; j0 < t.len; j0 += 32) f(t, t.off + j0 + lane, j0 + lane < t.len);
    }
    const unsigned c1 = *reinterpret_cast<volatile unsigned*>(&L.cnt[1]);
    for (unsigned i = blockIdx.x; i < c1; i += gridDim.x) {
        const RowTask t = L.t[1][i];
        for (int32_t j0 = warp * 32; j0 < t.len; j0 += kTierThreads) f(t, t.off + j0 + lane, j0 + lane < t.len);
    }
    // grid tier: the rows' 32-entry chunks are dealt round-robin to the warps
    // across all rows, so every warp stays busy whatever the row lengths
    const unsigned c2 = grid_tier ? *reinterpret_cast<volatile unsigned*>(&L.cnt[2]) : 0u;
    int64_t first = 0;                              // global index of the row's first chunk
    for (unsigned i = 0; i < c2; ++i) {
        const RowTask t = L.t[2][i];
        const int64_t nch = (static_cast<int64_t>(t.len) + 31) / 32;
        int64_t k = (static_cast<int64_t>(gw) - first) % static_cast<int64_t>(warps);
        if (k < 0) k += warps;
        for (; k < nch; k += warps) f(t, t.off + k * 32 + lane, k * 32 + lane < t.len);
        first += nch;
    }
}

// Runs every task filed in `L` (the functor sees each filed entry exactly
// once); with grid_tier false the caller handles the grid tier itself.
template <class F>
void run_tiers(const TierLists& L, const F& f, cudaStream_t s, bool grid_tier = true) {
    k_tiers<F><<<kTierGrid, kTierThreads, 0, s>>>(L, f, grid_tier);
}

// ----------------------------------------------------------------------------- dynamic adjacency

// Entry of an out-row that was deleted in place (rows are compacted when they
// move or when the store is rebuilt).
constexpr unsigned long long kRowTomb = ~0ull;

__host__ __device__ __forceinline__ unsigned long long pack_edge(int32_t label, int32_t target) {
    return (static_cast<unsigned long long>(static_cast<uint32_t>(label)) << 32) | static_cast<uint32_t>(target);
}

// The incremental path's adjacency: per vertex an out-row (packed label and
// target) and an in-row (sources), each with spare capacity so that a batch
// edits rows in place. In-rows are only appended to: an in-entry whose edge
// was deleted stays until the store is rebuilt, so in-rows name a superset of
// the current in-neighbours.
struct StoreView {
    int64_t* xro;
    int32_t* xlen;
    int32_t* xcap;
    unsigned long long* xpe;
    int64_t* yro;
    int32_t* ylen;
    int32_t* ycap;
    int32_t* ype;
};

}  // namespace bisim
