// Optional timing of the dominant (GEMM) kernel launches: when enabled, each
// GEMM kernel launch is bracketed by CUDA events on its own stream; the
// host reads the summed device time with mpgemm_profile_read().
#include <mutex>
#include <vector>

#include "common.cuh"
#include "profile.h"

namespace mpg {

static std::mutex g_pmu;
static int g_prof_on = 0;
static std::vector<cudaEvent_t> g_prof_ev;   // begin, end, begin, end, ...

ProfScope::ProfScope(cudaStream_t s) : s_(s), end_(nullptr) {
    std::lock_guard<std::mutex> lk(g_pmu);
    if (!g_prof_on) return;
    cudaEvent_t b;
    if (cudaEventCreate(&b) != cudaSuccess || cudaEventCreate(&end_) != cudaSuccess) {
        end_ = nullptr;
        return;
    }
    cudaEventRecord(b, s);
    g_prof_ev.push_back(b);
    g_prof_ev.push_back(end_);
}

ProfScope::~ProfScope() {
    if (end_) cudaEventRecord(end_, s_);
}

}  // namespace mpg

using namespace mpg;

extern "C" {

int mpgemm_profile(int enable) {
    std::lock_guard<std::mutex> lk(g_pmu);
    g_prof_on = enable ? 1 : 0;
    return MPGEMM_OK;
}

int mpgemm_profile_read(double* total_ms, int* launches) {
    std::vector<cudaEvent_t> ev;
    {
        std::lock_guard<std::mutex> lk(g_pmu);
        ev.swap(g_prof_ev);
    }
    double tot = 0.0;
    int n = 0, rc = MPGEMM_OK;
    for (size_t i = 0; i + 1 < ev.size(); i += 2) {
        float ms = 0.f;
        if (cudaEventSynchronize(ev[i + 1]) != cudaSuccess || cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) != cudaSuccess)
            rc = MPGEMM_ECUDA;
        tot += ms;
        n++;
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (total_ms) *total_ms = tot;
    if (launches) *launches = n;
    return rc;
}

}  // extern "C"
