// C ABI: nvd_graph_tune -- pick the work decomposition of the solve by timing it.
//
// The choices that decide how fast a PCG iteration (Section 3.2) runs on a given
// graph but not what it computes:
//   * tile width KT (k-blocking): how many right-hand sides share one SpMM; the
//     cost of k pairs is ceil(k / KT) tiles of one SpMM-driven solve each;
//   * row split: the light-row limit above which a row is split into heavy
//     sub-items (whole-row warp items or fixed-size chunks) instead of being
//     stored in the sliced layout, where it would make its whole slice as long;
//   * the number of light CTA blocks per SpMV launch;
//   * the gather engine of the multi-column SpMM (register slices, register stream,
//     TMA stream, asynchronous-copy stream);
//   * host-driven iterations versus one persistent cooperative launch per tile;
//   * two kernels per iteration (direction update folded into the SpMV) or three.
// Each candidate runs real solves on this graph with seeded synthetic
// right-hand sides (the structure decides the cost, not the values) for a fixed
// number of iterations; the cost of one iteration is the difference of two such
// runs divided by the difference of their iteration counts, so set-up and
// result collection cancel.  The search is coordinate-wise (tile width, row split,
// block count, launch mode, iteration form) and the winner is stored in the
// handle: later plans use it, and nvd_ge_distance uses the tile width and launch
// mode for the tuned solve mode when the caller leaves them open.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dispatch.h"
#include "solver.cuh"

using namespace nvd;

namespace {

// Seeded synthetic right-hand sides: x[j][i] in [0, 1) from a 64-bit mix of
// (i, j); y = 0.  Only the cost of the solve is measured with them.
__global__ void k_tune_rhs(double *x, int64_t n, int k) {
    const int64_t tot = n * k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = (uint64_t)t * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[t] = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    }
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    int init() {
        NVD_TRY_CUDA(cudaEventCreate(&a));
        NVD_TRY_CUDA(cudaEventCreate(&b));
        return NVD_OK;
    }
};

struct Bench {
    nvd_graph_s *g;
    int mode;              // solve mode actually timed (MIXED is timed as its FP32 inner solve)
    const double *x, *y;   // [32][n]
    double *d2;            // [32] device
    cudaStream_t s;
    Timer t;
    int lo, hi;            // iteration counts of the two runs

    bool fold = false;     // time the two-kernel iteration

    // One solve of KT columns, max_iter = iters; returns its device time in ms.
    int run(int KT, bool persistent, int iters, float *ms) {
        nvd_solve_opts o;
        nvd_solve_opts_default(&o);
        o.mode = mode;
        o.rtol = 1e-300;            // never met: every column runs max_iter iterations
        o.max_iter = iters;
        o.kt = KT;
        o.check_every = 4;
        o.flags = NVD_SOLVE_D2_DEVICE | (KT == 1 ? NVD_SOLVE_SINGLE_RHS : 0u) |
                  (persistent ? NVD_SOLVE_PERSISTENT : 0u) | (fold ? NVD_SOLVE_FOLD_DIRECTION : 0u);
        NVD_TRY_CUDA(cudaEventRecord(t.a, s));
        const int rc = ge_distance_internal(g, KT, x, y, NVD_F64, &o, d2, s);
        if (rc != NVD_OK && rc != NVD_ERR_NOT_CONVERGED) return rc;
        clear_error();
        NVD_TRY_CUDA(cudaEventRecord(t.b, s));
        NVD_TRY_CUDA(cudaEventSynchronize(t.b));
        NVD_TRY_CUDA(cudaEventElapsedTime(ms, t.a, t.b));
        return NVD_OK;
    }

    // Device time of one iteration of a KT-column tile (ms), best of two repeats.
    int per_iter(int KT, bool persistent, double *out) {
        float warm = 0.f;
        NVD_TRY(run(KT, persistent, lo, &warm));   // builds the plan, grows workspace
        double best = INFINITY;
        for (int rep = 0; rep < 2; ++rep) {
            float a = 0.f, b = 0.f;
            NVD_TRY(run(KT, persistent, lo, &a));
            NVD_TRY(run(KT, persistent, hi, &b));
            best = std::min(best, std::max(1e-6, (double)(b - a) / (hi - lo)));
        }
        *out = best;
        return NVD_OK;
    }
};

int tune_impl(nvd_graph_s *g, int32_t mode, int32_t k, uint32_t flags, nvd_tune_result *out, cudaStream_t s) {
    if (!g || mode < NVD_MODE_FP64 || mode > NVD_MODE_MIXED || k < 1 || (flags & ~NVD_TUNE_SINGLE_RHS)) {
        set_error("nvd_graph_tune: invalid argument (mode=%d k=%d flags=%u)", mode, k, flags);
        return NVD_ERR_INVALID_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != g->device) cudaSetDevice(g->device);
    struct Restore {
        int prev, dev;
        ~Restore() {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{prev, g->device};

    const bool single = flags & NVD_TUNE_SINGLE_RHS;
    int st = NVD_OK;
    double *x = (double *)g->wsp("tune_x", (size_t)32 * g->n * 8, &st);
    double *y = (double *)g->wsp("tune_y", (size_t)32 * g->n * 8, &st);
    double *d2 = (double *)g->wsp("tune_d2", 32 * 8, &st);
    if (st) return st;
    k_tune_rhs<<<(unsigned)std::min<int64_t>((32 * g->n + 255) / 256, 4096), 256, 0, s>>>(x, g->n, 32);
    NVD_TRY_CUDA(cudaGetLastError());
    NVD_TRY_CUDA(cudaMemsetAsync(y, 0, (size_t)32 * g->n * 8, s));

    Bench b{g, mode == NVD_MODE_MIXED ? (int)NVD_MODE_FP32 : (int)mode, x, y, d2, s, Timer(), 4, 12};
    NVD_TRY(b.t.init());
    const SpParams saved = g->sp;
    const int saved_kt = g->tuned_kt[mode], saved_pers = g->tuned_persistent[mode];
    const int saved_fold = g->tuned_fold[mode];
    g->tuned_kt[mode] = 0;
    g->tuned_persistent[mode] = 0;
    g->tuned_fold[mode] = 0;
    // the timed mode's own settings must not leak into the candidates (MIXED is
    // timed as FP32)
    const int tm = b.mode;
    const int keep_kt = g->tuned_kt[tm], keep_pers = g->tuned_persistent[tm], keep_fold = g->tuned_fold[tm];
    g->tuned_kt[tm] = 0;
    g->tuned_persistent[tm] = 0;
    g->tuned_fold[tm] = 0;
    auto restore_timed = [&]() {
        if (tm != mode) {
            g->tuned_kt[tm] = keep_kt;
            g->tuned_persistent[tm] = keep_pers;
            g->tuned_fold[tm] = keep_fold;
        }
    };
    auto fail = [&](int rc) {
        g->sp = saved;
        g->tuned_kt[mode] = saved_kt;
        g->tuned_persistent[mode] = saved_pers;
        g->tuned_fold[mode] = saved_fold;
        restore_timed();
        return rc;
    };

    // 1. tile width: minimise ceil(k / KT) * cost(KT)
    std::vector<int> kts = {1};
    if (!single)
        for (int c : {4, 8, 16, 32})
            if (c <= (b.mode == NVD_MODE_FP64 ? 16 : 32) && (c / 2 < k)) kts.push_back(c);
    g->sp = SpParams();
    int best_kt = 1;
    double best_cost = INFINITY, best_iter = INFINITY;
    int ntried = 0;
    for (int KT : kts) {
        double it = 0;
        int rc = b.per_iter(KT, false, &it);
        if (rc) return fail(rc);
        ++ntried;
        const double cost = std::ceil((double)k / KT) * it;
        if (cost < best_cost) {
            best_cost = cost;
            best_kt = KT;
            best_iter = it;
        }
    }
    // 2. row split, 3. light blocks per launch (each keeps the better of default and
    //    the candidates; the kept setting and the candidate are re-timed back to
    //    back, twice each, and the candidate must win by 2%: single timings differ
    //    by a few percent from run to run)
    for (int pass = 0; pass < 2; ++pass) {
        // fewer, larger blocks (25%) balance the fixed warp runs of multi-column
        // tiles better, and at four CTAs per SM fill one wave of 608 blocks
        std::vector<int> pcts = {50, 200};
        if (pass == 1 && best_kt > 1) pcts.insert(pcts.begin(), 25);
        for (int pct : pcts) {
            SpParams cand = g->sp;
            (pass == 0 ? cand.row_max_pct : cand.blocks_pct) = pct;
            const SpParams keep = g->sp;
            double base = INFINITY, alt = INFINITY;
            for (int rep = 0; rep < 2; ++rep) {
                double it = 0;
                g->sp = keep;
                int rc = b.per_iter(best_kt, false, &it);
                if (rc) return fail(rc);
                base = std::min(base, it);
                g->sp = cand;
                rc = b.per_iter(best_kt, false, &it);
                if (rc) return fail(rc);
                alt = std::min(alt, it);
            }
            ++ntried;
            if (alt < base * 0.98) {
                best_iter = alt;
            } else {
                g->sp = keep;
                best_iter = std::min(best_iter, base);
            }
        }
    }
    // 3b. gathers of the multi-column SpMM: register slices (default), register stream
    //     and, where the tile width allows it, TMA and asynchronous-copy streams
    if (best_kt > 1) {
        std::vector<int> modes = {0, 1};
        if (tma_tile(best_kt, b.mode == NVD_MODE_FP64 ? 8 : 4)) {
            modes.push_back(2);
            modes.push_back(3);
        }
        for (int gmode : modes) {
            if (gmode == g->sp.gather) continue;
            SpParams cand = g->sp;
            cand.gather = gmode;
            const SpParams keep = g->sp;
            double base = INFINITY, alt = INFINITY;
            for (int rep = 0; rep < 2; ++rep) {
                double it = 0;
                g->sp = keep;
                int rc = b.per_iter(best_kt, false, &it);
                if (rc) return fail(rc);
                base = std::min(base, it);
                g->sp = cand;
                rc = b.per_iter(best_kt, false, &it);
                if (rc) return fail(rc);
                alt = std::min(alt, it);
            }
            ++ntried;
            if (alt < base * 0.98) {
                best_iter = alt;
            } else {
                g->sp = keep;
                best_iter = std::min(best_iter, base);
            }
        }
    }
    // 4. one persistent launch per tile (not for the mixed mode, whose outer loop
    //    runs on the host)
    int pers = 0;
    if (mode != NVD_MODE_MIXED) {
        double it = 0, base = best_iter, alt = INFINITY;
        int rc = b.per_iter(best_kt, true, &it);
        if (rc == NVD_OK) {
            alt = it;
            // re-time both back to back before switching (as for the steps above)
            rc = b.per_iter(best_kt, false, &it);
            if (rc) return fail(rc);
            base = std::min(base, it);
            rc = b.per_iter(best_kt, true, &it);
            if (rc) return fail(rc);
            alt = std::min(alt, it);
            ++ntried;
            if (alt < base * 0.97) {
                pers = 1;
                best_iter = alt;
            } else {
                best_iter = base;
            }
        } else if (rc == NVD_ERR_UNSUPPORTED) {
            clear_error();   // does not fit one wave: host-driven only
        } else {
            return fail(rc);
        }
    }
    // 5. two kernels per iteration (direction folded into the SpMV) against three.
    //    The two forms are within a few percent of each other on many graphs, so
    //    both are re-timed back to back (twice each) and the folded form must win
    //    by 3%.
    int fold = 0;
    {
        double base = INFINITY, alt = INFINITY;
        for (int rep = 0; rep < 2; ++rep) {
            double it = 0;
            int rc = b.per_iter(best_kt, pers != 0, &it);
            if (rc) return fail(rc);
            base = std::min(base, it);
            b.fold = true;
            rc = b.per_iter(best_kt, pers != 0, &it);
            b.fold = false;
            if (rc) return fail(rc);
            alt = std::min(alt, it);
        }
        ++ntried;
        if (alt < base * 0.97) {
            fold = 1;
            best_iter = alt;
        } else {
            best_iter = std::min(best_iter, base);
        }
    }
    restore_timed();
    // drop the plans of the losing candidates
    for (auto it = g->plans.begin(); it != g->plans.end();) {
        const SpParams &p = it->second->sp;
        if (p.row_max_pct != g->sp.row_max_pct || p.blocks_pct != g->sp.blocks_pct || p.gather != g->sp.gather)
            it = g->plans.erase(it);
        else ++it;
    }
    g->tuned_kt[mode] = single ? 0 : best_kt;
    g->tuned_persistent[mode] = pers;
    g->tuned_fold[mode] = fold;
    if (out) {
        out->kt = best_kt;
        out->row_max_pct = g->sp.row_max_pct;
        out->blocks_pct = g->sp.blocks_pct;
        out->persistent = pers;
        out->candidates = ntried;
        out->fold_direction = fold;
        out->gather = g->sp.gather;
        out->l2_hot = g->sp.l2_hot;
        out->ms_per_iter = best_iter;
        out->ms_per_pair_iter = best_iter / best_kt;
    }
    return NVD_OK;
}

}  // namespace

extern "C" int nvd_graph_set_tuning(nvd_graph_t g, int32_t mode, const nvd_tune_result *t) {
    clear_error();
    if (!g || !t || mode < NVD_MODE_FP64 || mode > NVD_MODE_MIXED ||
        !(t->kt == 0 || t->kt == 1 || t->kt == 4 || t->kt == 8 || t->kt == 16 || t->kt == 32) ||
        t->row_max_pct < 10 || t->row_max_pct > 1000 || t->blocks_pct < 10 || t->blocks_pct > 1000 ||
        (t->persistent != 0 && t->persistent != 1) || (t->fold_direction != 0 && t->fold_direction != 1) ||
        t->gather < 0 || t->gather > 3 || (t->l2_hot != 0 && t->l2_hot != 1)) {
        set_error("nvd_graph_set_tuning: invalid argument");
        return NVD_ERR_INVALID_ARG;
    }
    g->sp.row_max_pct = t->row_max_pct;
    g->sp.blocks_pct = t->blocks_pct;
    g->sp.gather = t->gather;
    g->sp.l2_hot = t->l2_hot;
    g->tuned_kt[mode] = t->kt;
    g->tuned_persistent[mode] = t->persistent;
    g->tuned_fold[mode] = t->fold_direction;
    return NVD_OK;
}

extern "C" int nvd_graph_tune(nvd_graph_t g, int32_t mode, int32_t k, uint32_t flags, nvd_tune_result *out,
                              nvd_stream_t stream) {
    clear_error();
    TraceRange trace("nvd_graph_tune");
    try {
        return tune_impl(g, mode, k, flags, out, (cudaStream_t)stream);
    } catch (...) {
        set_error("nvd_graph_tune: unexpected host exception");
        return NVD_ERR_CUDA;
    }
}
