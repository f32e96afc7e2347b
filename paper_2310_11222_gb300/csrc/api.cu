// C ABI: status strings, defaults, version and the SpMV/SpMM launch timer.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <tuple>
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
    int cls;
    int64_t seq;     // SpMV launch number (class 0)
};
std::mutex g_mu;
int g_enabled = 0;   // 0 off, 1 SpMV launches, 2 SpMV and vector passes
int g_every = 1;     // time one SpMV launch in g_every
int64_t g_seq = 0;   // SpMV launches seen while enabled
std::vector<cudaEvent_t> g_pool;
std::vector<Pending> g_pending;
constexpr int NCLS = 3;   // 0 the CG SpMV/SpMM, 1 the vector passes, 2 the FP64 refinement residual SpMM
int64_t g_launches[NCLS] = {0, 0, 0};
double g_ms[NCLS] = {0.0, 0.0, 0.0}, g_bytes[NCLS] = {0.0, 0.0, 0.0};

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

size_t l2_persist_bytes() {
    static std::mutex mu;
    static std::vector<std::pair<int, size_t>> done;   // device, usable window bytes
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    for (const auto &d : done)
        if (d.first == dev) return d.second;
    int persist = 0, window = 0;
    size_t use = 0;
    if (cudaDeviceGetAttribute(&persist, cudaDevAttrMaxPersistingL2CacheSize, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&window, cudaDevAttrMaxAccessPolicyWindowSize, dev) == cudaSuccess && persist > 0 &&
        window > 0 && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)persist) == cudaSuccess)
        use = std::min((size_t)persist, (size_t)window);
    cudaGetLastError();
    done.emplace_back(dev, use);
    return use;
}

int allow_dynamic_smem(const void *kern, int bytes) {
    static std::mutex mu;
    static std::vector<std::tuple<const void *, int, int>> done;   // kernel, device, bytes
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    for (const auto &d : done)
        if (std::get<0>(d) == kern && std::get<1>(d) == dev && std::get<2>(d) >= bytes) return NVD_OK;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaFuncSetAttribute(MaxDynamicSharedMemorySize, %d) failed: %s", bytes, cudaGetErrorString(e));
        return NVD_ERR_CUDA;
    }
    done.emplace_back(kern, dev, bytes);
    return NVD_OK;
}

bool prof_enabled() { return g_enabled != 0; }
bool prof_vec_enabled() { return g_enabled >= 2; }

size_t prof_mark() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_pending.size();
}

// Of the SpMV launches (class 0) recorded in [mark, end), keep those among the
// first `keep` launched since sequence number seq0; the later ones ran after
// convergence and found no work.  Vector-pass launches (class 1) and launches
// outside the range are all kept.
void prof_keep_range(size_t mark, size_t end, int64_t keep, int64_t seq0) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (mark > g_pending.size()) return;
    end = std::min(end, g_pending.size());
    std::vector<Pending> kept(g_pending.begin(), g_pending.begin() + mark);
    for (size_t i = mark; i < g_pending.size(); ++i) {
        Pending &p = g_pending[i];
        if (i >= end || p.cls != 0 || p.seq - seq0 < keep) {
            kept.push_back(p);
        } else {
            cudaEventSynchronize(p.b);
            g_pool.push_back(p.a);
            g_pool.push_back(p.b);
        }
    }
    g_pending.swap(kept);
}

int64_t prof_seq() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_seq;
}

bool prof_begin(cudaStream_t s, int cls) {
    std::lock_guard<std::mutex> lk(g_mu);
    int64_t seq = -1;
    if (cls == 0) {
        seq = g_seq++;
        if (seq % g_every != 0) return false;   // not sampled: no events, no PDL break
    }
    Pending p{take_event(), take_event(), 0.0, cls, seq};
    cudaEventRecord(p.a, s);
    g_pending.push_back(p);
    return true;
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
    const int mode = on <= 0 ? 0 : on & 0xff;
    g_enabled = mode == 0 ? 0 : mode == 1 ? 1 : 2;
    const int every = on > 0 ? (on >> 8) & 0xff : 0;
    g_every = every < 1 ? 1 : every;
    return NVD_OK;
}

extern "C" int nvd_profile_read(int32_t kernel_class, int64_t *launches, double *total_ms, double *bytes) {
    clear_error();
    if (kernel_class < 0 || kernel_class >= NCLS) {
        set_error("nvd_profile_read: unknown kernel class %d", kernel_class);
        return NVD_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (Pending &p : g_pending) {
        if (cudaEventSynchronize(p.b) == cudaSuccess) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                g_ms[p.cls] += ms;
                g_bytes[p.cls] += p.bytes;
                ++g_launches[p.cls];
            }
        }
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.clear();
    cudaGetLastError();
    const int k = kernel_class;
    if (launches) *launches = g_launches[k];
    if (total_ms) *total_ms = g_ms[k];
    if (bytes) *bytes = g_bytes[k];
    g_launches[k] = 0;
    g_ms[k] = 0.0;
    g_bytes[k] = 0.0;
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
    o->check_every = 4;
    o->kt = 0;
    o->flags = 0;
}

extern "C" const char *nvd_version(void) { return "nvd-gb300 0.1.0 (sm_103a)"; }

extern "C" int64_t nvd_kernel_launches(void) { return g_kernel_launches.load(); }
