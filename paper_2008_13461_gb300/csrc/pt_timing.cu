// Per-kernel timing of the library's launches (a measurement aid; see
// pt_kernel_timing in pt.h): CUDA events recorded on the launching stream
// before and after each kernel, resolved and summed per kernel name when
// the totals are read.
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "pt_common.cuh"
#include "pt_kernels.cuh"

namespace ptk {

namespace {

struct Pending {
    const char *name;
    cudaEvent_t a, b;
};

struct Total {
    const char *name;
    int64_t launches;
    double ms;
};

std::atomic<int> g_on{0};
std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
std::vector<Total> g_total;

cudaEvent_t take_event() {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_free.empty()) {
            cudaEvent_t e = g_free.back();
            g_free.pop_back();
            return e;
        }
    }
    cudaEvent_t e = nullptr;
    return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
}

// Resolves the recorded launches into the totals (caller holds g_mu).
void drain() {
    for (const Pending &q : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
            Total *t = nullptr;
            for (Total &x : g_total)
                if (strcmp(x.name, q.name) == 0) t = &x;
            if (!t) {
                g_total.push_back({q.name, 0, 0.0});
                t = &g_total.back();
            }
            t->launches += 1;
            t->ms += ms;
        }
        g_free.push_back(q.a);
        g_free.push_back(q.b);
    }
    g_pending.clear();
}

}  // namespace

KernelTimer::KernelTimer(const char *name, cudaStream_t s) : name_(name), s_(s), a_(nullptr) {
    if (!g_on.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    a_ = take_event();
    if (a_ && cudaEventRecord(a_, s) != cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_mu);
        g_free.push_back(a_);
        a_ = nullptr;
    }
}

KernelTimer::~KernelTimer() {
    if (!a_) return;
    cudaEvent_t b = take_event();
    std::lock_guard<std::mutex> lk(g_mu);
    if (b && cudaEventRecord(b, s_) == cudaSuccess) {
        g_pending.push_back({name_, a_, b});
    } else {
        g_free.push_back(a_);
        if (b) g_free.push_back(b);
    }
}

}  // namespace ptk

using namespace ptk;

extern "C" pt_status pt_kernel_timing(int32_t enable) {
    if (enable != 0 && enable != 1) return PT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (enable) {
        drain();
        g_total.clear();
    }
    g_on.store(enable, std::memory_order_relaxed);
    return PT_OK;
}

extern "C" int32_t pt_kernel_timing_read(pt_kernel_time *out, int32_t max_entries) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain();
    const int32_t n = (int32_t)g_total.size();
    for (int32_t i = 0; out && i < n && i < max_entries; i++) {
        memset(out[i].name, 0, sizeof out[i].name);
        strncpy(out[i].name, g_total[i].name, sizeof out[i].name - 1);
        out[i].launches = g_total[i].launches;
        out[i].total_ms = g_total[i].ms;
    }
    return n;
}
