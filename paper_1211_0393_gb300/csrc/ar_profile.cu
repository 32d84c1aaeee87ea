// Per-kernel-class device timing: while enabled, a CUDA event pair is recorded
// on the launch stream around every kernel the library launches, and
// ar_profile_end() sums the elapsed times per class.  Recording events between
// kernels removes the overlap of programmatic dependent launch, so a profiled
// run measures each kernel alone.

#include "ar_internal.cuh"

#include <atomic>
#include <mutex>
#include <vector>

namespace ar {
namespace {

struct Rec {
    int kind;
    unsigned launches;
    cudaEvent_t a, b;
};

// Scopes opened inside a recording scope on the same thread are not recorded:
// an interval that brackets several dependent launches is timed as a whole.
thread_local int g_depth = 0;

std::mutex g_mu;
std::atomic<bool> g_on{false};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

int prof_begin(int kind, cudaStream_t s, unsigned launches) {
    if (!g_on.load(std::memory_order_relaxed) || g_depth > 0) return -1;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return -1;                        // a captured graph is not timed kernel by kernel
    std::lock_guard<std::mutex> lock(g_mu);
    Rec r{kind, launches, get_event(), get_event()};
    cudaEventRecord(r.a, s);
    g_recs.push_back(r);
    ++g_depth;
    return (int)g_recs.size() - 1;
}

void prof_end(int idx, cudaStream_t s) {
    if (idx < 0) return;
    --g_depth;
    std::lock_guard<std::mutex> lock(g_mu);
    if (idx < (int)g_recs.size()) cudaEventRecord(g_recs[idx].b, s);
}

}  // namespace ar

using namespace ar;

extern "C" {

ar_status ar_profile_begin(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_recs.clear();
    g_on.store(true);
    return AR_OK;
}

ar_status ar_profile_end(double* ms, unsigned long long* launches, int nkinds) {
    if (nkinds < 0 || (nkinds > 0 && (!ms || !launches)))
        return fail(AR_ERR_INVALID_ARG, "ar_profile_end: bad output arrays");
    g_on.store(false);
    std::lock_guard<std::mutex> lock(g_mu);
    for (int k = 0; k < nkinds; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    ar_status st = AR_OK;
    for (const Rec& r : g_recs) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
            st = fail(AR_ERR_CUDA, "ar_profile_end: event timing failed");
        if (r.kind >= 0 && r.kind < nkinds) {
            ms[r.kind] += t;
            launches[r.kind] += r.launches;
        }
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    return st;
}

}  // extern "C"
