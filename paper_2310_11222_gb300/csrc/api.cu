// C ABI: status strings, defaults, version and the SpMV/SpMM launch timer.
#include <atomic>
#include <mutex>
#include <vector>

#include "graph.h"

namespace nvd {
const char *last_error();

// ------------------------------------------------------------------ launch timer
// While enabled, launch_spmm() brackets each SpMV/SpMM launch with two CUDA events
// on the launching stream; nvd_profile_read() waits for them and sums.
namespace {
struct Pending {
    cudaEvent_t a, b;
    double bytes;
};
std::mutex g_mu;
bool g_enabled = false;
std::vector<cudaEvent_t> g_pool;
std::vector<Pending> g_pending;
int64_t g_launches = 0;
double g_ms = 0.0, g_bytes = 0.0;

cudaEvent_t take_event() {
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

std::atomic<int64_t> g_kernel_launches{0};

void note_launch(int64_t n) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

bool prof_enabled() { return g_enabled; }

size_t prof_mark() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_pending.size();
}

// Keep the first `keep` SpMV launches recorded after `mark`; the rest ran after
// convergence and found no work.
void prof_keep(size_t mark, int64_t keep) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (mark > g_pending.size()) return;
    const size_t upto = mark + (size_t)(keep < 0 ? 0 : keep);
    if (upto >= g_pending.size()) return;
    for (size_t i = upto; i < g_pending.size(); ++i) {
        cudaEventSynchronize(g_pending[i].b);
        g_pool.push_back(g_pending[i].a);
        g_pool.push_back(g_pending[i].b);
    }
    g_pending.resize(upto);
}

void prof_begin(cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    Pending p{take_event(), take_event(), 0.0};
    cudaEventRecord(p.a, s);
    g_pending.push_back(p);
}

void prof_end(cudaStream_t s, double bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_pending.empty()) return;
    Pending &p = g_pending.back();
    cudaEventRecord(p.b, s);
    p.bytes = bytes;
}

}  // namespace nvd

using namespace nvd;

extern "C" int nvd_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_enabled = on != 0;
    return NVD_OK;
}

extern "C" int nvd_profile_read(int32_t kernel_class, int64_t *launches, double *total_ms, double *bytes) {
    clear_error();
    if (kernel_class != 0) {
        set_error("nvd_profile_read: unknown kernel class %d", kernel_class);
        return NVD_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (Pending &p : g_pending) {
        if (cudaEventSynchronize(p.b) == cudaSuccess) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                g_ms += ms;
                g_bytes += p.bytes;
                ++g_launches;
            }
        }
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.clear();
    cudaGetLastError();
    if (launches) *launches = g_launches;
    if (total_ms) *total_ms = g_ms;
    if (bytes) *bytes = g_bytes;
    g_launches = 0;
    g_ms = 0.0;
    g_bytes = 0.0;
    return NVD_OK;
}

extern "C" const char *nvd_status_string(int status) {
    switch (status) {
        case NVD_OK: return "NVD_OK";
        case NVD_ERR_INVALID_ARG: return "NVD_ERR_INVALID_ARG";
        case NVD_ERR_NOT_SYMMETRIC: return "NVD_ERR_NOT_SYMMETRIC";
        case NVD_ERR_BAD_WEIGHT: return "NVD_ERR_BAD_WEIGHT";
        case NVD_ERR_OOM: return "NVD_ERR_OOM";
        case NVD_ERR_CUDA: return "NVD_ERR_CUDA";
        case NVD_ERR_NOT_CONVERGED: return "NVD_ERR_NOT_CONVERGED";
        case NVD_ERR_NUMERIC: return "NVD_ERR_NUMERIC";
        case NVD_ERR_TIMEOUT: return "NVD_ERR_TIMEOUT";
        case NVD_ERR_UNSUPPORTED: return "NVD_ERR_UNSUPPORTED";
    }
    return "NVD_ERR_UNKNOWN";
}

extern "C" const char *nvd_last_error(void) { return nvd::last_error(); }

extern "C" void nvd_solve_opts_default(nvd_solve_opts *o) {
    if (!o) return;
    o->mode = NVD_MODE_FP64;
    o->max_iter = 10000;
    o->rtol = 1e-10;
    o->d2_rtol = 1e-8;
    o->max_refine = 8;
    o->check_every = 8;
    o->kt = 0;
    o->flags = 0;
}

extern "C" const char *nvd_version(void) { return "nvd-gb300 0.1.0 (sm_103a)"; }

extern "C" int64_t nvd_kernel_launches(void) { return g_kernel_launches.load(); }
