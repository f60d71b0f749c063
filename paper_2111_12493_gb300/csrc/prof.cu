// Launch accounting and optional per-site kernel timing.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "bisim.h"
#include "prof.cuh"

namespace bisim {

namespace {

struct Pending {
    int site;
    cudaEvent_t start, stop;
    int64_t vertices, edges;
    double bytes;
};

struct Site {
    std::string name;
    int64_t launches = 0;
    double ms = 0.0, bytes = 0.0;
    int64_t vertices = 0, edges = 0;
};

std::mutex g_mu;
std::vector<Site> g_sites;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free_events;
std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_enabled{false};

cudaEvent_t take_event() {
    if (!g_free_events.empty()) {
        cudaEvent_t e = g_free_events.back();
        g_free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Resolves every recorded pair (waits for the events); caller holds g_mu.
void drain_locked() {
    for (const Pending& p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.stop) == cudaSuccess && cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
            Site& s = g_sites[p.site];
            s.launches += 1;
            s.ms += ms;
            s.bytes += p.bytes;
            s.vertices += p.vertices;
            s.edges += p.edges;
        }
        cudaGetLastError();
        g_free_events.push_back(p.start);
        g_free_events.push_back(p.stop);
    }
    g_pending.clear();
}

}  // namespace

int prof_site(const char* name) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t i = 0; i < g_sites.size(); ++i)
        if (g_sites[i].name == name) return static_cast<int>(i);
    g_sites.push_back(Site{name});
    return static_cast<int>(g_sites.size() - 1);
}

bool prof_enabled() { return g_enabled.load(std::memory_order_relaxed); }

void prof_add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void prof_add_bytes(int site, double bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (site >= 0 && site < static_cast<int>(g_sites.size())) g_sites[site].bytes += bytes;
}

void prof_add_work(int site, int64_t vertices, int64_t edges) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (site >= 0 && site < static_cast<int>(g_sites.size())) {
        g_sites[site].vertices += vertices;
        g_sites[site].edges += edges;
    }
}

Launch::Launch(int site, cudaStream_t s, int64_t vertices, int64_t edges, double alg_bytes)
    : site_(site), s_(s), vertices_(vertices), edges_(edges), bytes_(alg_bytes) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_enabled.load(std::memory_order_relaxed)) {
        std::lock_guard<std::mutex> lk(g_mu);
        start_ = take_event();
        cudaEventRecord(start_, s_);
    }
}

Launch::~Launch() {
    if (start_ == nullptr) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t stop = take_event();
    cudaEventRecord(stop, s_);
    g_pending.push_back(Pending{site_, start_, stop, vertices_, edges_, bytes_});
    if (g_pending.size() > 4096) drain_locked();
}

}  // namespace bisim

extern "C" {

void bisim_profile_enable(int32_t enable) { bisim::g_enabled.store(enable != 0); }

void bisim_profile_reset(void) {
    std::lock_guard<std::mutex> lk(bisim::g_mu);
    bisim::drain_locked();
    for (auto& s : bisim::g_sites) {
        s.launches = 0;
        s.ms = s.bytes = 0.0;
        s.vertices = s.edges = 0;
    }
}

int32_t bisim_profile_read(bisim_kernel_profile* out, int32_t max) {
    std::lock_guard<std::mutex> lk(bisim::g_mu);
    bisim::drain_locked();
    const int32_t n = static_cast<int32_t>(bisim::g_sites.size());
    for (int32_t i = 0; i < n && i < max && out != nullptr; ++i) {
        const auto& s = bisim::g_sites[i];
        std::memset(&out[i], 0, sizeof(out[i]));
        std::strncpy(out[i].name, s.name.c_str(), sizeof(out[i].name) - 1);
        out[i].launches = s.launches;
        out[i].total_ms = s.ms;
        out[i].alg_bytes = s.bytes;
        out[i].vertices = s.vertices;
        out[i].edges = s.edges;
    }
    return n;
}

int64_t bisim_launch_count(void) { return bisim::g_launches.load(); }

}  // extern "C"
