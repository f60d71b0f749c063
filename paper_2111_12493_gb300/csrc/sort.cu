// Device-wide exclusive scan and stable LSD radix sort (key u32, value u64).
//
// The radix sort is the classic three-phase scheme per 8-bit digit: per-tile
// digit histograms, one exclusive scan over the (digit, tile) counts, and a
// stable scatter in which every tile ranks its items with warp match masks.
#include <string>

#include "common.cuh"
#include "prof.cuh"

namespace bisim {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;   // 4096

constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 16;
constexpr int kRadixTile = kRadixThreads * kRadixItems;  // 4096
constexpr int kRadixBins = 256;
constexpr int kRadixWarps = kRadixThreads / 32;

__device__ __forceinline__ int64_t warp_inclusive_scan(int64_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Scans one tile of kScanTile values; writes the exclusive prefix within the
// tile and the tile total to block_sums[blockIdx.x].
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const int64_t* __restrict__ in,
                                                            int64_t* __restrict__ out, int64_t n,
                                                            int64_t* __restrict__ block_sums) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile +
                         static_cast<int64_t>(threadIdx.x) * kScanItems;
    int64_t v[kScanItems];
    int64_t run = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        run += v[i];
    }
    int64_t inc = warp_inclusive_scan(run);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t t = warp_tot[lane];
        int64_t ti = warp_inclusive_scan(t);
        warp_tot[lane] = ti - t;   // exclusive per warp
    }
    __syncthreads();
    int64_t excl = warp_tot[warp] + inc - run;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = excl;
        excl += v[i];
    }
    if (threadIdx.x == kScanThreads - 1) block_sums[blockIdx.x] = excl;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ offs) {
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / kScanTile];
}

__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                               int64_t m, int shift,
                                                               int64_t* __restrict__ counts,
                                                               int64_t ntiles) {
    __shared__ unsigned hist[kRadixBins];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kRadixTile;
#pragma unroll 4
    for (int r = 0; r < kRadixItems; ++r) {
        int64_t idx = base + static_cast<int64_t>(r) * kRadixThreads + threadIdx.x;
        if (idx < m) atomicAdd(&hist[(keys[idx] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    counts[static_cast<int64_t>(threadIdx.x) * ntiles + blockIdx.x] = hist[threadIdx.x];
}

// Stable scatter: items are visited in original order (round r, then thread),
// and each gets base[digit] + (earlier items of the tile with that digit).
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(
    const uint32_t* __restrict__ kin, const uint64_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint64_t* __restrict__ vout, int64_t m, int shift, const int64_t* __restrict__ offs,
    int64_t ntiles) {
    __shared__ int64_t base[kRadixBins];
    __shared__ unsigned running[kRadixBins];
    __shared__ unsigned wcnt[kRadixWarps][kRadixBins + 1];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    base[tid] = offs[static_cast<int64_t>(tid) * ntiles + blockIdx.x];
    running[tid] = 0;
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) wcnt[w][tid] = 0;
    if (tid < kRadixWarps) wcnt[tid][kRadixBins] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t tbase = static_cast<int64_t>(blockIdx.x) * kRadixTile;
    for (int r = 0; r < kRadixItems; ++r) {
        int64_t idx = tbase + static_cast<int64_t>(r) * kRadixThreads + tid;
        bool valid = idx < m;
        uint32_t k = valid ? kin[idx] : 0u;
        uint64_t v = valid ? vin[idx] : 0ull;
        unsigned d = valid ? ((k >> shift) & 0xffu) : static_cast<unsigned>(kRadixBins);
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned wrank = __popc(peers & lt);
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            unsigned pre = running[d];
            for (int w = 0; w < warp; ++w) pre += wcnt[w][d];
            int64_t pos = base[d] + pre + wrank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        unsigned tot = 0;
#pragma unroll
        for (int w = 0; w < kRadixWarps; ++w) {
            tot += wcnt[w][tid];
            wcnt[w][tid] = 0;
        }
        running[tid] += tot;
        __syncthreads();
    }
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Inputs of at most kSmallSortMax pairs (update batches, small frontiers): one
// CTA sorts (key bits, input index) composites by a bitonic network in shared
// memory, which is stable by construction and costs one launch instead of
// three per 8-bit digit.
constexpr int kSmallSortMax = 4096;
constexpr int kSmallSortThreads = 1024;

__global__ void __launch_bounds__(kSmallSortThreads) k_small_sort(const uint32_t* __restrict__ k0,
                                                                  const uint64_t* __restrict__ v0,
                                                                  uint32_t* __restrict__ k1, uint64_t* __restrict__ v1,
                                                                  int m, int p, uint32_t kmask) {
    __shared__ unsigned long long c[kSmallSortMax];
    for (int i = threadIdx.x; i < p; i += kSmallSortThreads)
        c[i] = i < m ? (static_cast<unsigned long long>(k0[i] & kmask) << 32) | static_cast<unsigned>(i) : ~0ull;
    __syncthreads();
    for (int k = 2; k <= p; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < p; i += kSmallSortThreads) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long a = c[i], b = c[l];
                    const bool up = (i & k) == 0;
                    if (up ? a > b : a < b) {
                        c[i] = b;
                        c[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < m; i += kSmallSortThreads) {
        const unsigned idx = static_cast<unsigned>(c[i]);
        k1[i] = k0[idx];
        v1[i] = v0[idx];
    }
}

}  // namespace

size_t scan_temp_words(int64_t n) {
    size_t words = 0;
    while (n > 1) {
        int64_t nb = cdiv(n, kScanTile);
        words += static_cast<size_t>(2 * nb);   // block sums and their scan
        n = nb;
    }
    return words + 2;
}

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s) {
    if (n <= 0) return;
    int64_t nb = cdiv(n, kScanTile);
    int64_t* sums = tmp;
    int64_t* sums_scan = tmp + nb;
    BISIM_SITE(site, "scan");
    {
        Launch L(site, s, 0, 0, 16.0 * n);
        k_scan_tile<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(in, out, n, sums);
    }
    if (nb > 1) {
        exclusive_scan_i64(sums, sums_scan, nb, tmp + 2 * nb, s);
        Launch L(site, s, 0, 0, 16.0 * n);
        k_scan_add<<<static_cast<unsigned>(cdiv(n, 256)), 256, 0, s>>>(out, n, sums_scan);
    }
}

size_t radix_temp_words(int64_t m) {
    int64_t ntiles = cdiv(m > 0 ? m : 1, kRadixTile);
    int64_t nc = ntiles * kRadixBins;
    return static_cast<size_t>(2 * nc) + scan_temp_words(nc);
}

int radix_sort_pairs(uint32_t* k0, uint64_t* v0, uint32_t* k1, uint64_t* v1, int64_t m, int bits,
                     int64_t* tmp, cudaStream_t s, const char* site_name) {
    if (m <= 0 || bits <= 0) return 0;
    if (m <= kSmallSortMax) {
        int p = 64;
        while (p < m) p <<= 1;
        const uint32_t kmask = bits >= 32 ? ~0u : ((1u << bits) - 1u);
        BISIM_SITE(site_small, "small_sort");
        Launch L(site_small, s, 0, m, 24.0 * m);
        k_small_sort<<<1, kSmallSortThreads, 0, s>>>(k0, v0, k1, v1, static_cast<int>(m), p, kmask);
        return 1;
    }
    const int64_t ntiles = cdiv(m, kRadixTile);
    const int64_t nc = ntiles * kRadixBins;
    int64_t* counts = tmp;
    int64_t* offs = tmp + nc;
    int64_t* stmp = tmp + 2 * nc;
    int which = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        const uint32_t* ki = which ? k1 : k0;
        const uint64_t* vi = which ? v1 : v0;
        uint32_t* ko = which ? k0 : k1;
        uint64_t* vo = which ? v0 : v1;
        // the site's passes are timed apart from other callers' (the CSR build's
        // full-size passes are the ones the benchmark's roofline names)
        const std::string name = site_name ? site_name : "radix";
        const int site_h = prof_site((name + "_hist").c_str());
        const int site_s = prof_site((name + "_scatter").c_str());
        {
            Launch L(site_h, s, 0, m, 4.0 * m);
            k_radix_hist<<<static_cast<unsigned>(ntiles), kRadixThreads, 0, s>>>(ki, m, shift, counts, ntiles);
        }
        exclusive_scan_i64(counts, offs, nc, stmp, s);
        Launch L(site_s, s, 0, m, 24.0 * m);
        k_radix_scatter<<<static_cast<unsigned>(ntiles), kRadixThreads, 0, s>>>(ki, vi, ko, vo, m, shift,
                                                                               offs, ntiles);
        which ^= 1;
    }
    return which;
}

}  // namespace bisim
