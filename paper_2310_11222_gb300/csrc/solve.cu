// C ABI: nvd_ge_distance and nvd_laplacian_apply.
//
// nvd_ge_distance evaluates the GE distance of Section 3.1,
//   d^2 = (x - y)^T L^+ (x - y),
// through a Laplacian solve (Section 3.2) instead of the pseudoinverse: pairs are
// processed in tiles of KT right-hand sides that share one SpMM per CG
// iteration, each (component, pair) keeping its own CG scalars.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <unordered_map>
#include <vector>

#include "dispatch.h"
#include "solver.cuh"

using namespace nvd;

// gather: dst[i] = src[perm[i]] (user -> internal); scatter: dst[perm[i]] = src[i].
template <class T>
__global__ void k_permute(const T *__restrict__ src, T *__restrict__ dst, const int32_t *__restrict__ perm,
                          int64_t n, bool gather) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (gather) dst[i] = src[perm[i]];
        else dst[perm[i]] = src[i];
    }
}

static int permute_vector(const void *src, void *dst, const int32_t *perm, int64_t n, int dtype, bool gather,
                   cudaStream_t s) {
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    if (dtype == NVD_F64)
        k_permute<double><<<grid, 256, 0, s>>>((const double *)src, (double *)dst, perm, n, gather);
    else
        k_permute<float><<<grid, 256, 0, s>>>((const float *)src, (float *)dst, perm, n, gather);
    note_launch();
    NVD_TRY_CUDA(cudaGetLastError());
    return NVD_OK;
}

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Tile width: explicit (opts.kt), else the tuner's choice for this mode (no wider
// than the pairs need), else the widest tile up to the pairs (FP64: 16, FP32: 32).
int pick_kt(const nvd_graph_s *g, const nvd_solve_opts &o, int k) {
    if (o.flags & NVD_SOLVE_SINGLE_RHS) return 1;
    if (o.kt) return o.kt;
    const int cap = g->tuned_kt[o.mode] ? g->tuned_kt[o.mode] : o.mode == NVD_MODE_FP64 ? 16 : 32;
    int kt = 1;
    for (int c : {4, 8, 16, 32})
        if (kt < k && c <= cap) kt = c;
    return k == 1 ? 1 : kt;
}

int check_opts(const nvd_solve_opts &o) {
    const uint32_t known = NVD_SOLVE_SINGLE_RHS | NVD_SOLVE_D2_DEVICE | NVD_SOLVE_HOST_INPUTS |
                           NVD_SOLVE_PERSISTENT | NVD_SOLVE_NO_SYNC | NVD_SOLVE_FOLD_DIRECTION |
                           NVD_SOLVE_TEST_TIMEOUT | NVD_SOLVE_D2_STOP | NVD_SOLVE_ELIMINATE;
    const bool d2stop = (o.flags & NVD_SOLVE_D2_STOP) != 0;
    if (o.mode < NVD_MODE_FP64 || o.mode > NVD_MODE_MIXED || !(o.rtol > 0.0) || o.max_iter < 1 ||
        o.check_every < 1 || !(o.kt == 0 || o.kt == 1 || o.kt == 4 || o.kt == 8 || o.kt == 16 || o.kt == 32) ||
        (o.flags & ~known) || (o.mode == NVD_MODE_MIXED && (!(o.d2_rtol > 0.0) || o.max_refine < 1)) ||
        (d2stop && (o.mode == NVD_MODE_MIXED || !(o.d2_rtol > 0.0) || !(o.d2_rtol < 1.0)))) {
        set_error("nvd_solve_opts: invalid field (mode=%d rtol=%g max_iter=%d check_every=%d kt=%d flags=%u)",
                  o.mode, o.rtol, o.max_iter, o.check_every, o.kt, o.flags);
        return NVD_ERR_INVALID_ARG;
    }
    return NVD_OK;
}

// idx: x, y are [k] device int32 node ids (indicator pairs e_x - e_y); the caller
// has checked them; host inputs and device d^2 are not used (z_out, if given, is
// [k][n] of xdt).
int distance_impl(nvd_graph_t g, int32_t k, const void *x, const void *y, int32_t xdt,
                  const nvd_solve_opts *opts, double *d2_out, void *z_out, nvd_solve_stats *stats,
                  cudaStream_t s, bool idx = false, const void *z0 = nullptr) {
    if (!g || k < 0 || (xdt != NVD_F32 && xdt != NVD_F64)) {
        set_error("nvd_ge_distance: invalid argument");
        return NVD_ERR_INVALID_ARG;
    }
    if (k == 0) return NVD_OK;
    TraceRange trace(idx ? "nvd solve (node-id pairs)" : "nvd_ge_distance");
    if (!x || !y || !d2_out) {
        set_error("nvd_ge_distance: x, y and d2_out are required");
        return NVD_ERR_INVALID_ARG;
    }
    nvd_solve_opts o;
    if (opts) o = *opts; else nvd_solve_opts_default(&o);
    NVD_TRY(check_opts(o));
    if (g->tuned_fold[o.mode]) o.flags |= NVD_SOLVE_FOLD_DIRECTION;
    if (z0 && (o.mode != NVD_MODE_FP64 || (o.flags & NVD_SOLVE_HOST_INPUTS) || idx)) {
        set_error("nvd_ge_distance_warm: a warm start needs FP64 mode and device inputs");
        return NVD_ERR_INVALID_ARG;
    }
    DeviceGuard guard(g->device);
    const int KT = pick_kt(g, o, k);
    const bool mixed = o.mode == NVD_MODE_MIXED;
    const size_t szv = o.mode == NVD_MODE_FP64 ? 8 : 4;
    const size_t xsz = xdt == NVD_F64 ? 8 : 4;
    const bool host_in = o.flags & NVD_SOLVE_HOST_INPUTS;
    const bool d2_dev = o.flags & NVD_SOLVE_D2_DEVICE;
    // persistent single-launch solve (FP64/FP32 modes; the launch timer needs the host
    // loop); it runs the register-path SpMM, so it takes a plan laid out for that
    const bool persistent = ((o.flags & NVD_SOLVE_PERSISTENT) || g->tuned_persistent[o.mode]) && !mixed &&
                            !prof_enabled() && !z0;
    Plan *pl = nullptr, *pl64 = nullptr;
    NVD_TRY(get_plan(g, KT, (int)szv, (int)szv, &pl, !persistent));
    if (mixed) NVD_TRY(get_plan(g, KT, 8, 8, &pl64));
    Ctx c;
    memset(&c, 0, sizeof(c));
    fill_graph_ctx(g, pl, &c);
    SolveWs w;
    NVD_TRY(setup_ws(g, pl, KT, szv, mixed, 1, &c, &w, s));
    if (mixed) {
        // the FP32 and FP64 plans share the slots and split-row sums
        NVD_TRY(setup_part(g, std::max(pl->part_slots(), pl64->part_slots()), KT, &c, &w, s));
        int st = NVD_OK;
        w.hsum = (double *)g->wsp("hsum", (size_t)std::max<int64_t>({pl->n_chunks, pl64->n_chunks, 1}) * KT * 8, &st);
        if (st) return st;
        c.hsum = w.hsum;
    }
    const int64_t sk = (int64_t)std::max(g->nseg, 1) * KT;
    unsigned *bar = nullptr;
    if (persistent) {
        int st = NVD_OK;
        bar = (unsigned *)g->wsp("bar", 16, &st);
        if (st) return st;
        c.bar_count = bar;
        c.bar_gen = bar + 1;
        c.bar_extra = (o.flags & NVD_SOLVE_TEST_TIMEOUT) ? 1 : 0;
    }
    // staging for host inputs/outputs: two slots, the next tile's copy on the copy
    // stream overlaps the current tile's solve
    void *sx[2] = {nullptr, nullptr}, *sy[2] = {nullptr, nullptr}, *sz = nullptr;
    const int32_t ntiles = (k + KT - 1) / KT;
    if (host_in) {
        int st = NVD_OK;
        const size_t tb = (size_t)KT * g->n * xsz;
        for (int q = 0; q < (ntiles > 1 ? 2 : 1); ++q) {
            sx[q] = g->wsp(q ? "stage_x1" : "stage_x", tb, &st);
            sy[q] = g->wsp(q ? "stage_y1" : "stage_y", tb, &st);
        }
        if (z_out) sz = g->wsp("stage_z", tb, &st);
        if (st) return st;
        if (!g->copy_stream) {
            NVD_TRY_CUDA(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking));
            for (int q = 0; q < 2; ++q) {
                NVD_TRY_CUDA(cudaEventCreateWithFlags(&g->ev_copied[q], cudaEventDisableTiming));
                NVD_TRY_CUDA(cudaEventCreateWithFlags(&g->ev_used[q], cudaEventDisableTiming));
            }
        }
        // the copy stream must not run ahead of work the caller queued on s before
        // this call (it may still write x, y)
        NVD_TRY_CUDA(cudaEventRecord(g->ev_used[1], s));
        NVD_TRY_CUDA(cudaStreamWaitEvent(g->copy_stream, g->ev_used[1], 0));
    }
    auto stage = [&](int32_t t) -> int {
        const int q = t & 1;
        const int32_t t0 = t * KT;
        const int kc = std::min<int>(KT, k - t0);
        const size_t off = (size_t)t0 * g->n * xsz;
        cudaStream_t cs = g->copy_stream;
        if (t >= 2) NVD_TRY_CUDA(cudaStreamWaitEvent(cs, g->ev_used[q], 0));
        NVD_TRY_CUDA(cudaMemcpyAsync(sx[q], (const char *)x + off, (size_t)kc * g->n * xsz, cudaMemcpyHostToDevice, cs));
        NVD_TRY_CUDA(cudaMemcpyAsync(sy[q], (const char *)y + off, (size_t)kc * g->n * xsz, cudaMemcpyHostToDevice, cs));
        NVD_TRY_CUDA(cudaEventRecord(g->ev_copied[q], cs));
        return NVD_OK;
    };
    // per-tile results stay on the device until the end of the call (no host sync
    // between tiles)
    int st_res = NVD_OK;
    ColResult *res_dev = (ColResult *)g->wsp("res_all", (size_t)ntiles * KT * sizeof(ColResult), &st_res);
    if (st_res) return st_res;
    std::vector<ColResult> res((size_t)ntiles * KT);
    std::vector<std::vector<int>> it_mixed(ntiles);
    std::vector<std::vector<double>> rr_mixed(ntiles);
    std::vector<int> steps_t(ntiles, 0), conv_t(ntiles, 1);
    std::vector<size_t> marks(ntiles, 0);
    std::vector<int64_t> seq0(ntiles, 0);
    int overall = NVD_OK;
    const bool need_host = !d2_dev || stats || host_in;
    if (host_in) NVD_TRY(stage(0));
    for (int32_t c0 = 0; c0 < k; c0 += KT) {
        const int32_t t = c0 / KT;
        const int kc = std::min<int>(KT, k - c0);
        const size_t off = (size_t)c0 * g->n * xsz;
        TraceRange trace_tile("nvd tile");
        TileIO io;
        io.kc = kc;
        if (host_in) {
            if (t + 1 < ntiles) NVD_TRY(stage(t + 1));
            NVD_TRY_CUDA(cudaStreamWaitEvent(s, g->ev_copied[t & 1], 0));
            io.x = sx[t & 1];
            io.y = sy[t & 1];
            io.z = sz;
        } else if (idx) {
            io.x = (const int32_t *)x + c0;
            io.y = (const int32_t *)y + c0;
            io.z = z_out ? (char *)z_out + off : nullptr;
            io.idx = 1;
        } else {
            io.x = (const char *)x + off;
            io.y = (const char *)y + off;
            io.z = z_out ? (char *)z_out + off : nullptr;
            io.z0 = z0 ? (const char *)z0 + off : nullptr;
        }
        if (io.z && g->n_singleton > 0)
            NVD_TRY_CUDA(cudaMemsetAsync(io.z, 0, (size_t)kc * g->n * xsz, s));
        // the tile's single owner: every segment of the graph, kc valid columns
        c.own0 = Owner{io.x, io.y, io.z, 0, g->n, kc, 0, g->nseg, io.idx};
        c.owners = nullptr;
        c.n_owner = 1;
        c.rtol2 = o.rtol * o.rtol;
        c.d2stop = (o.flags & NVD_SOLVE_D2_STOP) ? o.d2_rtol : 0.0;
        c.max_iter = o.max_iter;
        int steps = 0, conv = 1;
        marks[t] = prof_enabled() ? prof_mark() : 0;
        seq0[t] = prof_enabled() ? prof_seq() : 0;
        if (persistent) {
            // active, iters, status and n_active; the barrier's error flag (c.err)
            // stays sticky across the tiles of the call
            NVD_TRY_CUDA(cudaMemsetAsync(c.active, 0, (size_t)(3 * sk + 1) * 4, s));
            NVD_TRY_CUDA(cudaMemsetAsync(bar, 0, 16, s));
            PersistArgs a{w.delta, w.x, w.r, w.p, w.q, w.u, (o.flags & NVD_SOLVE_FOLD_DIRECTION) ? 1 : 0,
                          w.res, 1, io.z ? 1 : 0};
            NVD_TRY(run_persistent(g, c, a, o.mode, KT, xdt, s));
        } else if (o.mode == NVD_MODE_FP64)
            NVD_TRY(run_tile_fp64(g, c, w, o, io, s, KT, xdt));
        else if (o.mode == NVD_MODE_FP32)
            NVD_TRY(run_tile_fp32(g, c, w, o, io, s, KT, xdt));
        else
            NVD_TRY(run_tile_mixed(g, c, pl64, w, o, io, s, KT, xdt, it_mixed[t], rr_mixed[t], &steps, &conv));
        steps_t[t] = steps;
        conv_t[t] = conv;
        NVD_TRY(run_collect(c, KT, w.res, d2_dev ? d2_out + c0 : nullptr, 0, 1, s));
        NVD_TRY_CUDA(cudaMemcpyAsync(res_dev + (size_t)t * KT, w.res, KT * sizeof(ColResult),
                                     cudaMemcpyDeviceToDevice, s));
        if (host_in) NVD_TRY_CUDA(cudaEventRecord(g->ev_used[t & 1], s));
        if (host_in && z_out)
            NVD_TRY_CUDA(cudaMemcpyAsync((char *)z_out + off, sz, (size_t)kc * g->n * xsz, cudaMemcpyDeviceToHost, s));
    }
    if (need_host || prof_enabled()) {
        NVD_TRY_CUDA(cudaMemcpyAsync(res.data(), res_dev, (size_t)ntiles * KT * sizeof(ColResult),
                                     cudaMemcpyDeviceToHost, s));
        NVD_TRY_CUDA(cudaStreamSynchronize(s));
        if (prof_enabled() && !mixed) {
            // drop the post-convergence SpMV launches of each tile (last tile first:
            // the earlier marks stay valid)
            for (int32_t t = ntiles - 1; t >= 0; --t) {
                int real = 0;
                for (int j = 0; j < std::min<int>(KT, k - t * KT); ++j) real = std::max(real, res[(size_t)t * KT + j].iters);
                prof_keep_range(marks[t], t + 1 < ntiles ? marks[t + 1] : (size_t)-1, real, seq0[t]);
            }
        }
    }
    if (need_host) {
        for (int32_t t = 0; t < ntiles; ++t) {
            const int32_t c0 = t * KT;
            const int kc = std::min<int>(KT, k - c0);
            for (int j = 0; j < kc; ++j) {
                ColResult &r = res[(size_t)t * KT + j];
                if (mixed) r.status = conv_t[t] ? NVD_OK : NVD_ERR_NOT_CONVERGED;
                if (!d2_dev) d2_out[c0 + j] = r.d2;
                if (r.status != NVD_OK && overall != NVD_ERR_NUMERIC) overall = r.status;
                if (stats) {
                    nvd_solve_stats &st = stats[c0 + j];
                    st.status = r.status;
                    st.reserved = 0;
                    if (mixed) {
                        st.iters = it_mixed[t][j];
                        st.refine_steps = steps_t[t];
                        st.rel_resid = rr_mixed[t][j];
                    } else {
                        st.iters = r.iters;
                        st.refine_steps = 0;
                        st.rel_resid = r.rr0 > 0.0 ? std::sqrt(std::max(r.rr, 0.0) / r.rr0) : 0.0;
                    }
                }
            }
        }
    }
    if (persistent || !(o.flags & NVD_SOLVE_NO_SYNC) || need_host) {
        // a bounded device wait that gave up (the persistent kernel's grid barrier, a
        // TMA gather that never arrived) leaves its status in c.err
        int32_t err = 0;
        NVD_TRY_CUDA(cudaMemcpyAsync(&err, c.err, 4, cudaMemcpyDeviceToHost, s));
        NVD_TRY_CUDA(cudaStreamSynchronize(s));
        if (err != 0) {
            set_error("nvd_ge_distance: a bounded device wait gave up (status %d)", err);
            return err;
        }
    }
    if (!(o.flags & NVD_SOLVE_NO_SYNC) || need_host) NVD_TRY_CUDA(cudaStreamSynchronize(s));
    if (overall != NVD_OK) set_error("nvd_ge_distance: some pair ended with status %d (%s)", overall,
                                     nvd_status_string(overall));
    return overall;
}

// Effective resistance R(u, v) = (e_u - e_v)^T L^+ (e_u - e_v): pairs inside one
// component go to the solve as indicator pairs (the delta kernel builds e_u - e_v
// from the ids); u = v gives 0 and u, v in different components (or an isolated
// node) give +inf without a solve.
int resistance_impl(nvd_graph_t g, int32_t k, const int32_t *u, const int32_t *v, const nvd_solve_opts *opts,
                    double *r_out, nvd_solve_stats *stats, cudaStream_t s) {
    if (!g || k < 0) {
        set_error("nvd_effective_resistance: invalid argument");
        return NVD_ERR_INVALID_ARG;
    }
    if (k == 0) return NVD_OK;
    if (!u || !v || !r_out) {
        set_error("nvd_effective_resistance: u, v and r_out are required");
        return NVD_ERR_INVALID_ARG;
    }
    nvd_solve_opts o;
    if (opts) o = *opts; else nvd_solve_opts_default(&o);
    NVD_TRY(check_opts(o));
    if (o.flags & (NVD_SOLVE_D2_DEVICE | NVD_SOLVE_HOST_INPUTS)) {
        set_error("nvd_effective_resistance: NVD_SOLVE_D2_DEVICE and NVD_SOLVE_HOST_INPUTS do not apply "
                  "(ids and results are host arrays)");
        return NVD_ERR_INVALID_ARG;
    }
    std::vector<int32_t> su, sv;
    std::vector<int32_t> where;  // solved pair -> its index in [0, k)
    for (int32_t j = 0; j < k; ++j) {
        if (u[j] < 0 || u[j] >= g->n || v[j] < 0 || v[j] >= g->n) {
            set_error("nvd_effective_resistance: pair %d has a node id outside [0, %lld)", j, (long long)g->n);
            return NVD_ERR_INVALID_ARG;
        }
    }
    for (int32_t j = 0; j < k; ++j) {
        const int32_t a = g->h_seg_of[u[j]], b = g->h_seg_of[v[j]];
        const bool solve = u[j] != v[j] && a >= 0 && a == b;
        r_out[j] = u[j] == v[j] ? 0.0 : std::numeric_limits<double>::infinity();
        if (stats) stats[j] = nvd_solve_stats{0, 0, 0.0, NVD_OK, 0};
        if (solve) {
            su.push_back(u[j]);
            sv.push_back(v[j]);
            where.push_back(j);
        }
    }
    const int32_t m = (int32_t)su.size();
    if (m == 0) return NVD_OK;
    DeviceGuard guard(g->device);
    int st = NVD_OK;
    int32_t *ids = (int32_t *)g->wsp("resist_ids", (size_t)2 * m * 4, &st);
    if (st) return st;
    NVD_TRY_CUDA(cudaMemcpyAsync(ids, su.data(), (size_t)m * 4, cudaMemcpyHostToDevice, s));
    NVD_TRY_CUDA(cudaMemcpyAsync(ids + m, sv.data(), (size_t)m * 4, cudaMemcpyHostToDevice, s));
    std::vector<double> r(m);
    std::vector<nvd_solve_stats> sst(stats ? m : 0);
    const int rc = (o.flags & NVD_SOLVE_ELIMINATE)
                       ? elim_distance(g, m, ids, ids + m, NVD_F64, &o, r.data(), nullptr,
                                       stats ? sst.data() : nullptr, s, true)
                       : distance_impl(g, m, ids, ids + m, NVD_F64, &o, r.data(), nullptr,
                                       stats ? sst.data() : nullptr, s, true);
    if (rc != NVD_OK && rc != NVD_ERR_NOT_CONVERGED && rc != NVD_ERR_NUMERIC) return rc;
    for (int32_t i = 0; i < m; ++i) {
        r_out[where[i]] = r[i];
        if (stats) stats[where[i]] = sst[i];
    }
    if (rc != NVD_OK) set_error("nvd_effective_resistance: some pair ended with status %d (%s)", rc,
                                nvd_status_string(rc));
    return rc;
}

__global__ void k_gather_f64(const double *__restrict__ z, const int64_t *__restrict__ off, double *__restrict__ out,
                             int64_t m) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = z[off[t]];
}

__device__ __forceinline__ double pos_inf() { return __longlong_as_double(0x7ff0000000000000LL); }

// R[i][j] of the subset from the gathered solution entries.  Position i has node
// node[i], group q[i] (-1: isolated) and member a[i] of its group; member a >= 1 of
// group q is solve column col1[q] + a - 1, whose entries at the group's members
// start at zval[off[column]] (member order).  Z(a, b) = z_a at member b, 0 for the
// reference member 0; R = Z(a,a) - Z(a,b) - Z(b,a) + Z(b,b).
__global__ void k_rmat_assemble(int32_t s_n, const int32_t *__restrict__ node, const int32_t *__restrict__ q,
                                const int32_t *__restrict__ a, const int32_t *__restrict__ col1,
                                const int64_t *__restrict__ off, const double *__restrict__ zval,
                                double *__restrict__ R) {
    const int64_t tot = (int64_t)s_n * s_n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = (int32_t)(t / s_n), j = (int32_t)(t % s_n);
        double r;
        if (node[i] == node[j]) {
            r = 0.0;
        } else if (q[i] < 0 || q[i] != q[j]) {
            r = pos_inf();
        } else {
            const int32_t ai = a[i], bj = a[j], c1 = col1[q[i]];
            const double *za = ai ? zval + off[c1 + ai - 1] : nullptr;
            const double *zb = bj ? zval + off[c1 + bj - 1] : nullptr;
            const double zaa = za ? za[ai] : 0.0, zab = za ? za[bj] : 0.0;
            const double zba = zb ? zb[ai] : 0.0, zbb = zb ? zb[bj] : 0.0;
            r = zaa - zab - zba + zbb;
        }
        R[t] = r;
    }
}

// (1/2) sum_ij p_i p_j R_ij over the pairs with p_i p_j > 0 (+inf if one of them has
// R = inf): per-block partials in a fixed order, then one block adds them in block
// order, so the result does not depend on scheduling.
constexpr int QF_NT = 256;
__device__ __forceinline__ void qf_block_sum(double v, bool inf, double *sh, double *out, int *out_inf) {
    sh[threadIdx.x] = v;
    const int any = __syncthreads_or(inf ? 1 : 0);
    for (int w = QF_NT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *out = sh[0];
        *out_inf = any;
    }
}
__global__ void k_quadform_part(int32_t m, const double *__restrict__ p, const double *__restrict__ R,
                                double *__restrict__ part, int *__restrict__ part_inf) {
    __shared__ double sh[QF_NT];
    const int64_t tot = (int64_t)m * m;
    double acc = 0.0;
    bool inf = false;
    for (int64_t t = (int64_t)blockIdx.x * QF_NT + threadIdx.x; t < tot; t += (int64_t)gridDim.x * QF_NT) {
        const double w = p[t / m] * p[t % m];
        if (w > 0.0) {
            const double r = R[t];
            if (isinf(r)) inf = true;
            else acc += w * r;
        }
    }
    qf_block_sum(acc, inf, sh, part + blockIdx.x, part_inf + blockIdx.x);
}
__global__ void k_quadform_final(int32_t nb, const double *__restrict__ part, const int *__restrict__ part_inf,
                                 double *__restrict__ out) {
    __shared__ double sh[QF_NT];
    __shared__ int fl;
    double acc = 0.0;
    bool inf = false;
    for (int b = threadIdx.x; b < nb; b += QF_NT) {
        acc += part[b];
        inf = inf || part_inf[b] != 0;
    }
    qf_block_sum(acc, inf, sh, out, &fl);
    if (threadIdx.x == 0) out[0] = fl ? pos_inf() : 0.5 * out[0];
}

// Effective-resistance matrix on a node subset, left on the device in R_dev
// ([s][s]).  Per component, one reference node r and one solve per other distinct
// node d: z_d = L^+ (e_d - e_r) (z_r = 0).  By linearity z_a - z_b = L^+ (e_a - e_b),
// so
//   R(a, b) = (e_a - e_b)^T (z_a - z_b) = z_a[a] - z_a[b] - z_b[a] + z_b[b],
// which needs only the entries of every z at the subset's nodes of its component:
// they are gathered on the device after each batch of solves, and k_rmat_assemble
// forms R (0 on repeated nodes, +inf across components).
int resistance_matrix_core(nvd_graph_t g, int32_t s_n, const int32_t *nodes, const nvd_solve_opts &o,
                           double *R_dev, nvd_solve_stats *stats, cudaStream_t s) {
    for (int32_t i = 0; i < s_n; ++i)
        if (nodes[i] < 0 || nodes[i] >= g->n) {
            set_error("nvd_resistance_matrix: nodes[%d] is outside [0, %lld)", i, (long long)g->n);
            return NVD_ERR_INVALID_ARG;
        }
    // distinct nodes per segment, in first-seen order; the first is the reference
    std::vector<int32_t> seg_slot(g->nseg, -1);
    std::vector<std::vector<int32_t>> grp;   // distinct node ids
    std::vector<int32_t> pos_q(s_n, -1), pos_a(s_n, 0);
    {
        std::unordered_map<int32_t, int32_t> member;
        for (int32_t i = 0; i < s_n; ++i) {
            const int32_t sg = g->h_seg_of[nodes[i]];
            if (sg < 0) continue;
            if (seg_slot[sg] < 0) {
                seg_slot[sg] = (int32_t)grp.size();
                grp.emplace_back();
            }
            auto &G = grp[seg_slot[sg]];
            auto it = member.find(nodes[i]);
            if (it == member.end()) {
                it = member.emplace(nodes[i], (int32_t)G.size()).first;
                G.push_back(nodes[i]);
            }
            pos_q[i] = seg_slot[sg];
            pos_a[i] = it->second;
        }
    }
    // columns: member m >= 1 of group q is column col1[q] + m - 1 and solves
    // e_{G[m]} - e_{G[0]}; its gathered entries start at col_off[column]
    const int32_t ngrp = (int32_t)grp.size();
    std::vector<int32_t> su, sv, col_grp, col1(std::max(ngrp, 1), 0);
    std::vector<int64_t> col_off;
    int64_t nval = 0;
    for (int32_t q = 0; q < ngrp; ++q) {
        col1[q] = (int32_t)su.size();
        for (size_t m = 1; m < grp[q].size(); ++m) {
            su.push_back(grp[q][m]);
            sv.push_back(grp[q][0]);
            col_grp.push_back(q);
            col_off.push_back(nval);
            nval += (int64_t)grp[q].size();
        }
    }
    const int32_t ncol = (int32_t)su.size();
    TraceRange trace("nvd_resistance_matrix");
    if (stats) for (int32_t i = 0; i < s_n; ++i) stats[i] = nvd_solve_stats{0, 0, 0.0, NVD_OK, 0};
    DeviceGuard guard(g->device);
    int st = NVD_OK;
    // index tables: node, q, a [s_n] | col1 [ngrp] | ids u, v [ncol]  (int32), col_off [ncol] (int64)
    const size_t nint = (size_t)3 * s_n + col1.size() + 2 * (size_t)ncol;
    std::vector<int32_t> hint;
    hint.reserve(nint);
    hint.insert(hint.end(), nodes, nodes + s_n);
    hint.insert(hint.end(), pos_q.begin(), pos_q.end());
    hint.insert(hint.end(), pos_a.begin(), pos_a.end());
    hint.insert(hint.end(), col1.begin(), col1.end());
    hint.insert(hint.end(), su.begin(), su.end());
    hint.insert(hint.end(), sv.begin(), sv.end());
    int32_t *dint = (int32_t *)g->wsp("rmat_int", nint * 4, &st);
    int64_t *doff_col = (int64_t *)g->wsp("rmat_coloff", std::max<size_t>(col_off.size(), 1) * 8, &st);
    double *zval = (double *)g->wsp("rmat_zval", (size_t)std::max<int64_t>(nval, 1) * 8, &st);
    if (st) return st;
    NVD_TRY_CUDA(cudaMemcpyAsync(dint, hint.data(), nint * 4, cudaMemcpyHostToDevice, s));
    if (ncol) NVD_TRY_CUDA(cudaMemcpyAsync(doff_col, col_off.data(), col_off.size() * 8, cudaMemcpyHostToDevice, s));
    const int32_t *d_node = dint, *d_q = dint + s_n, *d_a = dint + 2 * s_n, *d_col1 = dint + 3 * s_n;
    const int32_t *ids_u = d_col1 + col1.size(), *ids_v = ids_u + ncol;
    int overall = NVD_OK;
    if (ncol > 0) {
        // columns per solve call: z of a batch is at most 2^28 doubles (2 GiB)
        const int32_t chunk = (int32_t)std::max<int64_t>(1, std::min<int64_t>(ncol, ((int64_t)1 << 28) / g->n));
        double *zb = (double *)g->wsp("rmat_z", (size_t)chunk * g->n * 8, &st);
        if (st) return st;
        std::vector<nvd_solve_stats> cst(ncol);
        std::vector<double> d2(chunk);
        for (int32_t c0 = 0; c0 < ncol; c0 += chunk) {
            const int32_t kc = std::min(chunk, ncol - c0);
            const int rc = distance_impl(g, kc, ids_u + c0, ids_v + c0, NVD_F64, &o, d2.data(), zb, cst.data() + c0,
                                         s, true);
            if (rc != NVD_OK && rc != NVD_ERR_NOT_CONVERGED && rc != NVD_ERR_NUMERIC) return rc;
            if (rc != NVD_OK && overall != NVD_ERR_NUMERIC) overall = rc;
            // offsets into zb of this batch's entries at the members of each column's group
            std::vector<int64_t> off;
            off.reserve((size_t)(kc ? (c0 + kc < ncol ? col_off[c0 + kc] : nval) - col_off[c0] : 0));
            for (int32_t c = c0; c < c0 + kc; ++c)
                for (int32_t v : grp[col_grp[c]]) off.push_back((int64_t)(c - c0) * g->n + v);
            const int64_t m = (int64_t)off.size();
            int64_t *doff = (int64_t *)g->wsp("rmat_off", (size_t)m * 8, &st);
            if (st) return st;
            NVD_TRY_CUDA(cudaMemcpyAsync(doff, off.data(), (size_t)m * 8, cudaMemcpyHostToDevice, s));
            k_gather_f64<<<(int)std::min<int64_t>((m + 255) / 256, 1024), 256, 0, s>>>(zb, doff, zval + col_off[c0],
                                                                                         m);
            note_launch();
            NVD_TRY_CUDA(cudaGetLastError());
            // the next batch overwrites zb and the offsets
            NVD_TRY_CUDA(cudaStreamSynchronize(s));
        }
        if (stats)
            for (int32_t i = 0; i < s_n; ++i)
                if (pos_q[i] >= 0 && pos_a[i] > 0) stats[i] = cst[col1[pos_q[i]] + pos_a[i] - 1];
    }
    const int64_t tot = (int64_t)s_n * s_n;
    k_rmat_assemble<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, s>>>(s_n, d_node, d_q, d_a, d_col1,
                                                                                     doff_col, zval, R_dev);
    note_launch();
    NVD_TRY_CUDA(cudaGetLastError());
    if (overall != NVD_OK) set_error("nvd_resistance_matrix: some solve ended with status %d (%s)", overall,
                                     nvd_status_string(overall));
    return overall;
}

int rmat_check(nvd_graph_t g, int32_t s_n, const nvd_solve_opts *opts, nvd_solve_opts *o, const char *who) {
    if (!g || s_n < 0) {
        set_error("%s: invalid argument", who);
        return NVD_ERR_INVALID_ARG;
    }
    if (opts) *o = *opts; else nvd_solve_opts_default(o);
    NVD_TRY(check_opts(*o));
    if (o->flags & (NVD_SOLVE_D2_DEVICE | NVD_SOLVE_HOST_INPUTS | NVD_SOLVE_D2_STOP)) {
        set_error("%s: NVD_SOLVE_D2_DEVICE, NVD_SOLVE_HOST_INPUTS and NVD_SOLVE_D2_STOP do not apply (host "
                  "arrays; entries are combinations of solutions, not d^2 values)", who);
        return NVD_ERR_INVALID_ARG;
    }
    return NVD_OK;
}

int resistance_matrix_impl(nvd_graph_t g, int32_t s_n, const int32_t *nodes, const nvd_solve_opts *opts,
                           double *R, nvd_solve_stats *stats, cudaStream_t s) {
    nvd_solve_opts o;
    NVD_TRY(rmat_check(g, s_n, opts, &o, "nvd_resistance_matrix"));
    if (s_n == 0) return NVD_OK;
    if (!nodes || !R) {
        set_error("nvd_resistance_matrix: nodes and R_out are required");
        return NVD_ERR_INVALID_ARG;
    }
    DeviceGuard guard(g->device);
    int st = NVD_OK;
    double *R_dev = (double *)g->wsp("rmat_R", (size_t)s_n * s_n * 8, &st);
    if (st) return st;
    const int rc = resistance_matrix_core(g, s_n, nodes, o, R_dev, stats, s);
    if (rc != NVD_OK && rc != NVD_ERR_NOT_CONVERGED && rc != NVD_ERR_NUMERIC) return rc;
    NVD_TRY_CUDA(cudaMemcpyAsync(R, R_dev, (size_t)s_n * s_n * 8, cudaMemcpyDeviceToHost, s));
    NVD_TRY_CUDA(cudaStreamSynchronize(s));
    return rc;
}

// Network variance of node weights p: (1/2) sum_ij p_i p_j R(i, j) over the nodes
// with p_i > 0, from the resistance matrix of that support (on the device).
int network_variance_impl(nvd_graph_t g, int32_t s_n, const int32_t *nodes, const double *p,
                          const nvd_solve_opts *opts, double *var_out, cudaStream_t s) {
    nvd_solve_opts o;
    NVD_TRY(rmat_check(g, s_n, opts, &o, "nvd_network_variance"));
    if (!var_out || (s_n > 0 && (!nodes || !p))) {
        set_error("nvd_network_variance: invalid argument");
        return NVD_ERR_INVALID_ARG;
    }
    std::vector<int32_t> sup;
    std::vector<double> ps;
    for (int32_t i = 0; i < s_n; ++i) {
        if (nodes[i] < 0 || nodes[i] >= g->n) {
            set_error("nvd_network_variance: nodes[%d] is outside [0, %lld)", i, (long long)g->n);
            return NVD_ERR_INVALID_ARG;
        }
        if (!(p[i] >= 0.0) || !std::isfinite(p[i])) {
            set_error("nvd_network_variance: p[%d] = %g is not a finite non-negative weight", i, p[i]);
            return NVD_ERR_INVALID_ARG;
        }
        if (p[i] > 0.0) {
            sup.push_back(nodes[i]);
            ps.push_back(p[i]);
        }
    }
    *var_out = 0.0;
    const int32_t m = (int32_t)sup.size();
    if (m == 0) return NVD_OK;
    DeviceGuard guard(g->device);
    int st = NVD_OK;
    const int64_t tot = (int64_t)m * m;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((tot + QF_NT * 16 - 1) / (QF_NT * 16), 1024));
    double *R_dev = (double *)g->wsp("rmat_R", (size_t)tot * 8, &st);
    double *dp = (double *)g->wsp("var_p", (size_t)m * 8 + (size_t)nb * 8 + 8, &st);
    int *dinf = (int *)g->wsp("var_inf", (size_t)nb * 4, &st);
    if (st) return st;
    double *part = dp + m, *dout = part + nb;
    NVD_TRY_CUDA(cudaMemcpyAsync(dp, ps.data(), (size_t)m * 8, cudaMemcpyHostToDevice, s));
    const int rc = resistance_matrix_core(g, m, sup.data(), o, R_dev, nullptr, s);
    if (rc != NVD_OK && rc != NVD_ERR_NOT_CONVERGED && rc != NVD_ERR_NUMERIC) return rc;
    k_quadform_part<<<nb, QF_NT, 0, s>>>(m, dp, R_dev, part, dinf);
    note_launch();
    NVD_TRY_CUDA(cudaGetLastError());
    k_quadform_final<<<1, QF_NT, 0, s>>>(nb, part, dinf, dout);
    note_launch();
    NVD_TRY_CUDA(cudaGetLastError());
    NVD_TRY_CUDA(cudaMemcpyAsync(var_out, dout, 8, cudaMemcpyDeviceToHost, s));
    NVD_TRY_CUDA(cudaStreamSynchronize(s));
    return rc;
}

int apply_impl(nvd_graph_t g, int32_t k, const void *x, void *y, int32_t dtype, cudaStream_t s) {
    if (!g || k < 0 || (k > 0 && (!x || !y)) || (dtype != NVD_F32 && dtype != NVD_F64)) {
        set_error("nvd_laplacian_apply: invalid argument");
        return NVD_ERR_INVALID_ARG;
    }
    if (k == 0) return NVD_OK;
    DeviceGuard guard(g->device);
    const size_t sz = dtype == NVD_F64 ? 8 : 4;
    Plan *pl = nullptr;
    NVD_TRY(get_plan(g, 1, (int)sz, (int)sz, &pl));
    Ctx c;
    memset(&c, 0, sizeof(c));
    fill_graph_ctx(g, pl, &c);
    if (dtype == NVD_F32) {
        const float *w32 = nullptr;
        NVD_TRY(get_w32(g, &w32, s));
        c.w = w32;
    }
    int st = NVD_OK;
    void *xin = nullptr, *yout = nullptr;
    if (g->perm.p) {
        xin = g->wsp("apply_x", g->n * sz, &st);
        yout = g->wsp("apply_y", g->n * sz, &st);
        if (st) return st;
    }
    NVD_TRY_CUDA(cudaMemsetAsync(y, 0, (size_t)k * g->n * sz, s));
    for (int32_t j = 0; j < k; ++j) {
        const char *xj = (const char *)x + (size_t)j * g->n * sz;
        char *yj = (char *)y + (size_t)j * g->n * sz;
        if (!g->perm.p) {
            NVD_TRY(run_apply(g, c, xj, yj, dtype, s));
        } else {
            NVD_TRY(permute_vector(xj, xin, g->perm.as<int32_t>(), g->n, dtype, true, s));
            NVD_TRY_CUDA(cudaMemsetAsync(yout, 0, g->n * sz, s));
            NVD_TRY(run_apply(g, c, xin, yout, dtype, s));
            NVD_TRY(permute_vector(yout, yj, g->perm.as<int32_t>(), g->n, dtype, false, s));
        }
    }
    NVD_TRY_CUDA(cudaStreamSynchronize(s));
    return NVD_OK;
}

}  // namespace

namespace nvd {
int ge_distance_internal(nvd_graph_t g, int32_t k, const void *x, const void *y, int32_t xdt,
                         const nvd_solve_opts *opts, double *d2_out, cudaStream_t s) {
    return distance_impl(g, k, x, y, xdt, opts, d2_out, nullptr, nullptr, s);
}
}  // namespace nvd

extern "C" int nvd_ge_distance(nvd_graph_t g, int32_t k, const void *x, const void *y, int32_t xdtype,
                               const nvd_solve_opts *opts, double *d2_out, void *z_out,
                               nvd_solve_stats *stats, nvd_stream_t stream) {
    clear_error();
    try {
        if (opts && (opts->flags & NVD_SOLVE_ELIMINATE)) {
            nvd_solve_opts o = *opts;
            NVD_TRY(check_opts(o));
            return elim_distance(g, k, x, y, xdtype, &o, d2_out, z_out, stats, (cudaStream_t)stream);
        }
        return distance_impl(g, k, x, y, xdtype, opts, d2_out, z_out, stats, (cudaStream_t)stream);
    } catch (const std::bad_alloc &) {
        set_error("nvd_ge_distance: host allocation failed");
        return NVD_ERR_OOM;
    } catch (...) {
        set_error("nvd_ge_distance: unexpected host exception");
        return NVD_ERR_CUDA;
    }
}

extern "C" int nvd_ge_distance_warm(nvd_graph_t g, int32_t k, const void *x, const void *y, int32_t xdtype,
                                    const void *z0, const nvd_solve_opts *opts, double *d2_out, void *z_out,
                                    nvd_solve_stats *stats, nvd_stream_t stream) {
    clear_error();
    if (k > 0 && !z0) {
        set_error("nvd_ge_distance_warm: z0 is required");
        return NVD_ERR_INVALID_ARG;
    }
    try {
        return distance_impl(g, k, x, y, xdtype, opts, d2_out, z_out, stats, (cudaStream_t)stream, false, z0);
    } catch (const std::bad_alloc &) {
        set_error("nvd_ge_distance_warm: host allocation failed");
        return NVD_ERR_OOM;
    } catch (...) {
        set_error("nvd_ge_distance_warm: unexpected host exception");
        return NVD_ERR_CUDA;
    }
}

extern "C" int nvd_effective_resistance(nvd_graph_t g, int32_t k, const int32_t *u, const int32_t *v,
                                        const nvd_solve_opts *opts, double *r_out, nvd_solve_stats *stats,
                                        nvd_stream_t stream) {
    clear_error();
    try {
        return resistance_impl(g, k, u, v, opts, r_out, stats, (cudaStream_t)stream);
    } catch (const std::bad_alloc &) {
        set_error("nvd_effective_resistance: host allocation failed");
        return NVD_ERR_OOM;
    } catch (...) {
        set_error("nvd_effective_resistance: unexpected host exception");
        return NVD_ERR_CUDA;
    }
}

extern "C" int nvd_resistance_matrix(nvd_graph_t g, int32_t s_n, const int32_t *nodes,
                                     const nvd_solve_opts *opts, double *R_out, nvd_solve_stats *stats,
                                     nvd_stream_t stream) {
    clear_error();
    try {
        return resistance_matrix_impl(g, s_n, nodes, opts, R_out, stats, (cudaStream_t)stream);
    } catch (const std::bad_alloc &) {
        set_error("nvd_resistance_matrix: host allocation failed");
        return NVD_ERR_OOM;
    } catch (...) {
        set_error("nvd_resistance_matrix: unexpected host exception");
        return NVD_ERR_CUDA;
    }
}

extern "C" int nvd_network_variance(nvd_graph_t g, int32_t s_n, const int32_t *nodes, const double *p,
                                    const nvd_solve_opts *opts, double *var_out, nvd_stream_t stream) {
    clear_error();
    try {
        return network_variance_impl(g, s_n, nodes, p, opts, var_out, (cudaStream_t)stream);
    } catch (const std::bad_alloc &) {
        set_error("nvd_network_variance: host allocation failed");
        return NVD_ERR_OOM;
    } catch (...) {
        set_error("nvd_network_variance: unexpected host exception");
        return NVD_ERR_CUDA;
    }
}

extern "C" int nvd_laplacian_apply(nvd_graph_t g, int32_t k, const void *x, void *y, int32_t dtype,
                                   nvd_stream_t stream) {
    clear_error();
    try {
        return apply_impl(g, k, x, y, dtype, (cudaStream_t)stream);
    } catch (...) {
        set_error("nvd_laplacian_apply: unexpected host exception");
        return NVD_ERR_CUDA;
    }
}
