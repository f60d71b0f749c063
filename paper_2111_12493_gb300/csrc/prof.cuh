// Launch accounting: a process-wide launch counter and optional event timing
// per launch site (see bisim_profile_* in bisim.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace bisim {

// Registers (once) and returns the index of a launch site.
int prof_site(const char* name);
// Whether launches are being timed (timed launches cannot sit in a captured graph).
bool prof_enabled();
// Adjusts the launch counter for kernels that run inside a graph replay.
void prof_add_launches(int64_t n);
// Adds algorithmic bytes to a site after its launches (work known only once they ran).
void prof_add_bytes(int site, double bytes);
// Adds the vertices and edges a site's launches processed, when only the device knew them.
void prof_add_work(int site, int64_t vertices, int64_t edges);

// Brackets one kernel launch: counts it and, when profiling is enabled,
// records events around it on stream `s`.
class Launch {
  public:
    Launch(int site, cudaStream_t s, int64_t vertices, int64_t edges, double alg_bytes);
    ~Launch();
    Launch(const Launch&) = delete;
    Launch& operator=(const Launch&) = delete;

  private:
    int site_;
    cudaStream_t s_;
    cudaEvent_t start_ = nullptr;
    int64_t vertices_, edges_;
    double bytes_;
};

}  // namespace bisim

// Declares a function-local static site id and brackets the statement that follows.
#define BISIM_SITE(var, name) static const int var = ::bisim::prof_site(name)
