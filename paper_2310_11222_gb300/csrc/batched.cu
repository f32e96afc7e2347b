// C ABI: nvd_ge_distance_batched -- many graphs in one solve.
//
// The G graphs are concatenated once into an internal union graph: the diagonal
// blocks of one block-diagonal Laplacian, graph g owning node range
// [off_g, off_g + n_g) and its own segments (connected components).  Every
// (graph, pair) keeps its own CG scalars and convergence test, so the result
// equals G separate solves.  One tile of pairs is solved by the host-driven
// loop of nvd_ge_distance over the union graph (every graph's rows in each
// launch, owners table for the inputs and results), or, with
// NVD_SOLVE_PERSISTENT, by one cooperative persistent kernel (persistent.cuh),
// captured in a CUDA graph together with its state resets and the copy of the
// results; repeated calls with the same arguments replay the captured graph.
#include <algorithm>
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <vector>

#include "dispatch.h"
#include "solver.cuh"

using namespace nvd;

namespace {

__global__ void k_shift_i64(int64_t *dst, const int64_t *src, int64_t n, int64_t add) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i] + add;
}
__global__ void k_shift_i32(int32_t *dst, const int32_t *src, int64_t n, int32_t add) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i] + add;
}
__global__ void k_iota_i32(int32_t *dst, int64_t n, int32_t add) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (int32_t)i + add;
}
__global__ void k_f32_to_f64(double *dst, const float *src, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

int grid_of(int64_t n, int sms) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 16)); }

struct Captured {
    cudaGraphExec_t exec = nullptr;
    ~Captured() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

struct UnionGraph {
    std::vector<uint64_t> ids;
    cudaStream_t cs = nullptr;        // capture/replay stream (the caller's may be the legacy stream)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::unique_ptr<nvd_graph_s> g;
    std::vector<int64_t> node_off;    // [G+1]
    std::vector<int32_t> seg_off;     // [G+1] segment range of each graph
    ColResult *h_res = nullptr;       // pinned, [G][32]
    size_t h_res_cap = 0;
    std::map<std::vector<uint64_t>, std::unique_ptr<Captured>> graphs;
    ~UnionGraph() {
        graphs.clear();
        if (h_res) cudaFreeHost(h_res);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (cs) cudaStreamDestroy(cs);
    }
};

std::mutex g_mu;
std::list<std::unique_ptr<UnionGraph>> g_cache;   // most recent first, at most 4

int build_union(const nvd_graph_t *gs, int G, cudaStream_t s, UnionGraph **out) {
    std::unique_ptr<UnionGraph> u(new UnionGraph());
    u->g.reset(new nvd_graph_s());
    nvd_graph_s *U = u->g.get();
    U->id = next_graph_id();
    U->device = gs[0]->device;
    U->num_sms = gs[0]->num_sms;
    bool all_f32 = true;
    int64_t n = 0, nnz = 0;
    u->node_off.assign(G + 1, 0);
    u->seg_off.assign(G + 1, 0);
    for (int i = 0; i < G; ++i) {
        u->ids.push_back(gs[i]->id);
        if (gs[i]->wdtype != NVD_F32) all_f32 = false;
        u->node_off[i + 1] = u->node_off[i] + gs[i]->n;
        u->seg_off[i + 1] = u->seg_off[i] + gs[i]->nseg;
        n += gs[i]->n;
        nnz += gs[i]->nnz;
    }
    if (n > INT32_MAX - 1) {
        set_error("nvd_ge_distance_batched: %lld nodes in total exceed 2^31", (long long)n);
        return NVD_ERR_INVALID_ARG;
    }
    U->n = n;
    U->nnz = nnz;
    U->nnz_user = nnz;
    U->wdtype = all_f32 ? NVD_F32 : NVD_F64;
    const size_t wsz = all_f32 ? 4 : 8;
    const int64_t npad = ((nnz + 3) / 4) * 4 + 4;
    NVD_TRY(U->rowptr.alloc((n + 1) * 8));
    NVD_TRY(U->colidx.alloc(npad * 4));
    NVD_TRY(U->w.alloc(npad * wsz));
    NVD_TRY_CUDA(cudaMemsetAsync(U->colidx.p, 0, npad * 4, s));
    NVD_TRY_CUDA(cudaMemsetAsync(U->w.p, 0, npad * wsz, s));
    NVD_TRY(U->deg64.alloc(n * 8));
    NVD_TRY(U->dinv64.alloc(n * 8));
    NVD_TRY(U->deg32.alloc(n * 4));
    NVD_TRY(U->dinv32.alloc(n * 4));
    bool any_perm = false;
    for (int i = 0; i < G; ++i) any_perm = any_perm || gs[i]->perm.p;
    if (any_perm) NVD_TRY(U->perm.alloc(n * 4));
    U->h_rowptr.assign(n + 1, 0);
    int64_t eoff = 0;
    for (int i = 0; i < G; ++i) {
        const nvd_graph_s *g = gs[i];
        const int64_t no = u->node_off[i];
        k_shift_i64<<<grid_of(g->n, U->num_sms), 256, 0, s>>>(U->rowptr.as<int64_t>() + no, g->rowptr.as<int64_t>(),
                                                             g->n, eoff);
        if (g->nnz)
            k_shift_i32<<<grid_of(g->nnz, U->num_sms), 256, 0, s>>>(U->colidx.as<int32_t>() + eoff,
                                                                   g->colidx.as<int32_t>(), g->nnz, (int32_t)no);
        if (g->nnz) {
            if (all_f32 || g->wdtype == NVD_F64)
                NVD_TRY_CUDA(cudaMemcpyAsync((char *)U->w.p + eoff * wsz, g->w.p, g->nnz * wsz,
                                             cudaMemcpyDeviceToDevice, s));
            else
                k_f32_to_f64<<<grid_of(g->nnz, U->num_sms), 256, 0, s>>>(U->w.as<double>() + eoff, g->w.as<float>(),
                                                                        g->nnz);
        }
        NVD_TRY_CUDA(cudaMemcpyAsync(U->deg64.as<double>() + no, g->deg64.p, g->n * 8, cudaMemcpyDeviceToDevice, s));
        NVD_TRY_CUDA(cudaMemcpyAsync(U->dinv64.as<double>() + no, g->dinv64.p, g->n * 8, cudaMemcpyDeviceToDevice, s));
        NVD_TRY_CUDA(cudaMemcpyAsync(U->deg32.as<float>() + no, g->deg32.p, g->n * 4, cudaMemcpyDeviceToDevice, s));
        NVD_TRY_CUDA(cudaMemcpyAsync(U->dinv32.as<float>() + no, g->dinv32.p, g->n * 4, cudaMemcpyDeviceToDevice, s));
        if (any_perm) {
            if (g->perm.p)
                k_shift_i32<<<grid_of(g->n, U->num_sms), 256, 0, s>>>(U->perm.as<int32_t>() + no, g->perm.as<int32_t>(),
                                                                     g->n, (int32_t)no);
            else
                k_iota_i32<<<grid_of(g->n, U->num_sms), 256, 0, s>>>(U->perm.as<int32_t>() + no, g->n, (int32_t)no);
        }
        for (int64_t r = 0; r < g->n; ++r) U->h_rowptr[no + r] = g->h_rowptr[r] + eoff;
        for (int sg = 0; sg < g->nseg; ++sg) {
            U->h_seg_begin.push_back(g->h_seg_begin[sg] + no);
            U->h_seg_end.push_back(g->h_seg_end[sg] + no);
        }
        U->ncomp += g->ncomp;
        U->n_singleton += g->n_singleton;
        eoff += g->nnz;
    }
    U->h_rowptr[n] = nnz;
    const int64_t last = nnz;
    NVD_TRY_CUDA(cudaMemcpyAsync(U->rowptr.as<int64_t>() + n, &last, 8, cudaMemcpyHostToDevice, s));
    NVD_TRY_CUDA(cudaGetLastError());
    U->nseg = (int32_t)U->h_seg_begin.size();
    const size_t ns = std::max<size_t>(U->nseg, 1);
    NVD_TRY(U->seg_begin.alloc(ns * 8));
    NVD_TRY(U->seg_end.alloc(ns * 8));
    NVD_TRY(U->seg_owner.alloc(ns * 4));
    std::vector<int32_t> owner(ns, 0);
    for (int i = 0; i < G; ++i)
        for (int sg = u->seg_off[i]; sg < u->seg_off[i + 1]; ++sg) owner[sg] = i;
    if (U->nseg) {
        NVD_TRY_CUDA(cudaMemcpyAsync(U->seg_begin.p, U->h_seg_begin.data(), U->nseg * 8, cudaMemcpyHostToDevice, s));
        NVD_TRY_CUDA(cudaMemcpyAsync(U->seg_end.p, U->h_seg_end.data(), U->nseg * 8, cudaMemcpyHostToDevice, s));
    }
    NVD_TRY_CUDA(cudaMemcpyAsync(U->seg_owner.p, owner.data(), ns * 4, cudaMemcpyHostToDevice, s));
    NVD_TRY_CUDA(cudaStreamCreateWithFlags(&u->cs, cudaStreamNonBlocking));
    NVD_TRY_CUDA(cudaEventCreateWithFlags(&u->ev_in, cudaEventDisableTiming));
    NVD_TRY_CUDA(cudaEventCreateWithFlags(&u->ev_out, cudaEventDisableTiming));
    NVD_TRY_CUDA(cudaStreamSynchronize(s));
    *out = u.release();
    return NVD_OK;
}

int get_union(const nvd_graph_t *gs, int G, cudaStream_t s, UnionGraph **out) {
    std::vector<uint64_t> ids(G);
    for (int i = 0; i < G; ++i) ids[i] = gs[i]->id;
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_cache.begin(); it != g_cache.end(); ++it)
        if ((*it)->ids == ids) {
            g_cache.splice(g_cache.begin(), g_cache, it);
            *out = g_cache.front().get();
            return NVD_OK;
        }
    UnionGraph *u = nullptr;
    NVD_TRY(build_union(gs, G, s, &u));
    g_cache.emplace_front(u);
    while (g_cache.size() > 4) g_cache.pop_back();
    *out = u;
    return NVD_OK;
}

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

int batched_impl(const nvd_graph_t *gs, int32_t G, const int32_t *k_per, const void *const *x,
                 const void *const *y, int32_t xdt, const nvd_solve_opts *opts, double *d2_out,
                 nvd_solve_stats *stats, cudaStream_t s) {
    if (!gs || G < 1 || !k_per || !x || !y || !d2_out || (xdt != NVD_F32 && xdt != NVD_F64)) {
        set_error("nvd_ge_distance_batched: invalid argument");
        return NVD_ERR_INVALID_ARG;
    }
    int kmax = 0;
    int64_t ktot = 0;
    for (int i = 0; i < G; ++i) {
        if (!gs[i] || k_per[i] < 0 || (k_per[i] > 0 && (!x[i] || !y[i])) || gs[i]->device != gs[0]->device) {
            set_error("nvd_ge_distance_batched: invalid graph %d", i);
            return NVD_ERR_INVALID_ARG;
        }
        kmax = std::max(kmax, k_per[i]);
        ktot += k_per[i];
    }
    if (ktot == 0) return NVD_OK;
    nvd_solve_opts o;
    if (opts) o = *opts; else nvd_solve_opts_default(&o);
    if (o.mode == NVD_MODE_MIXED) {
        set_error("nvd_ge_distance_batched: the MIXED mode is not available for batches");
        return NVD_ERR_UNSUPPORTED;
    }
    if (!(o.rtol > 0.0) || o.max_iter < 1 || !(o.kt == 0 || o.kt == 1 || o.kt == 4 || o.kt == 8 || o.kt == 16 ||
                                                 o.kt == 32)) {
        set_error("nvd_ge_distance_batched: invalid options");
        return NVD_ERR_INVALID_ARG;
    }
    DeviceGuard guard(gs[0]->device);
    UnionGraph *u = nullptr;
    NVD_TRY(get_union(gs, G, s, &u));
    nvd_graph_s *U = u->g.get();
    int KT = o.kt;
    if (!KT) {
        const int cap = o.mode == NVD_MODE_FP64 ? 16 : 32;
        KT = 1;
        for (int cnd : {4, 8, 16, 32})
            if (KT < kmax && cnd <= cap) KT = cnd;
        if (kmax == 1) KT = 1;
    }
    const size_t szv = o.mode == NVD_MODE_FP64 ? 8 : 4;
    const size_t xsz = xdt == NVD_F64 ? 8 : 4;
    Plan *pl = nullptr;
    NVD_TRY(get_plan(U, KT, (int)szv, (int)szv, &pl, false));   // the persistent kernel's register-path SpMM
    Ctx c;
    memset(&c, 0, sizeof(c));
    fill_graph_ctx(U, pl, &c);
    SolveWs w;
    NVD_TRY(setup_ws(U, pl, KT, szv, false, G, &c, &w, s));
    int st = NVD_OK;
    unsigned *bar = (unsigned *)U->wsp("bar", 16, &st);
    Owner *d_own = (Owner *)U->wsp("owners", (size_t)G * sizeof(Owner), &st);
    if (st) return st;
    c.bar_count = bar;
    c.bar_gen = bar + 1;
    c.owners = d_own;
    c.n_owner = G;
    c.rtol2 = o.rtol * o.rtol;
    c.max_iter = o.max_iter;
    if (u->h_res_cap < (size_t)G * KT) {
        if (u->h_res) cudaFreeHost(u->h_res);
        u->h_res = nullptr;
        NVD_TRY_CUDA(cudaHostAlloc((void **)&u->h_res, (size_t)G * KT * sizeof(ColResult), cudaHostAllocDefault));
        u->h_res_cap = (size_t)G * KT;
    }
    if (o.mode == NVD_MODE_FP32) {
        const float *w32 = nullptr;   // create the FP32 weights before any capture
        NVD_TRY(get_w32(U, &w32, s));
    }
    PersistArgs a{w.delta, w.x, w.r, w.p, w.q, w.u, (o.flags & NVD_SOLVE_FOLD_DIRECTION) ? 1 : 0, w.res, G, 0};
    const int64_t sk = (int64_t)std::max(U->nseg, 1) * KT;
    int overall = NVD_OK;
    std::vector<int64_t> out_off(G + 1, 0);
    for (int i = 0; i < G; ++i) out_off[i + 1] = out_off[i] + k_per[i];
    for (int c0 = 0; c0 < kmax; c0 += KT) {
        std::vector<Owner> own(G);
        for (int i = 0; i < G; ++i) {
            const int kc = std::max(0, std::min(KT, k_per[i] - c0));
            const int64_t ng = gs[i]->n;
            own[i] = Owner{kc ? (const char *)x[i] + (size_t)c0 * ng * xsz : nullptr,
                           kc ? (const char *)y[i] + (size_t)c0 * ng * xsz : nullptr, nullptr, u->node_off[i], ng,
                           kc, u->seg_off[i], u->seg_off[i + 1], 0};
        }
        if (!(o.flags & NVD_SOLVE_PERSISTENT)) {
            // the same phases as separate launches over the union graph, on the
            // caller's stream, every graph's rows in each launch
            NVD_TRY_CUDA(cudaMemcpyAsync(d_own, own.data(), G * sizeof(Owner), cudaMemcpyHostToDevice, s));
            NVD_TRY_CUDA(cudaMemsetAsync(c.active, 0, (size_t)(3 * sk + 8) * 4, s));
            TileIO io{};
            io.owners = true;
            io.kc = KT;
            const int rc = o.mode == NVD_MODE_FP64 ? run_tile_fp64(U, c, w, o, io, s, KT, xdt)
                                                   : run_tile_fp32(U, c, w, o, io, s, KT, xdt);
            if (rc != NVD_OK && rc != NVD_ERR_NOT_CONVERGED) return rc;
            NVD_TRY(run_collect(c, KT, w.res, nullptr, 0, G, s));
            NVD_TRY_CUDA(cudaMemcpyAsync(u->h_res, w.res, (size_t)G * KT * sizeof(ColResult), cudaMemcpyDeviceToHost,
                                         s));
            NVD_TRY_CUDA(cudaStreamSynchronize(s));
        } else {
            // one persistent launch, captured with its resets and result copy; the
            // key holds everything the captured launch depends on
            std::vector<uint64_t> key = {(uint64_t)KT, (uint64_t)o.mode, (uint64_t)xdt, (uint64_t)c0,
                                         (uint64_t)o.max_iter, (uint64_t)pl->n_sblk, (uint64_t)a.fold};
            uint64_t rbits;
            memcpy(&rbits, &o.rtol, 8);
            key.push_back(rbits);
            // workspace addresses: a regrown workspace is a new key
            for (const void *ptr : {(const void *)w.part, (const void *)w.gpart, (const void *)w.gcount,
                                    (const void *)w.x, (const void *)w.r, (const void *)w.p, (const void *)w.q,
                                    (const void *)a.u, (const void *)w.delta, (const void *)w.res,
                                    (const void *)c.active, (const void *)w.hsum, (const void *)c.rho,
                                    (const void *)bar, (const void *)d_own})
                key.push_back((uint64_t)(uintptr_t)ptr);
            for (int i = 0; i < G; ++i) {
                key.push_back((uint64_t)(uintptr_t)own[i].x);
                key.push_back((uint64_t)(uintptr_t)own[i].y);
                key.push_back((uint64_t)own[i].kc);
            }
            auto &cap = u->graphs[key];
            // order the library stream after the caller's work
            NVD_TRY_CUDA(cudaEventRecord(u->ev_in, s));
            NVD_TRY_CUDA(cudaStreamWaitEvent(u->cs, u->ev_in, 0));
            cudaStream_t cs = u->cs;
            NVD_TRY_CUDA(cudaMemcpyAsync(d_own, own.data(), G * sizeof(Owner), cudaMemcpyHostToDevice, cs));
            if (!cap) {
                NVD_TRY_CUDA(cudaStreamSynchronize(cs));
                std::unique_ptr<Captured> cp(new Captured());
                cudaGraph_t graph = nullptr;
                NVD_TRY_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
                int rc = NVD_OK;
                if (cudaMemsetAsync(c.active, 0, (size_t)(3 * sk + 8) * 4, cs) != cudaSuccess ||
                    cudaMemsetAsync(bar, 0, 16, cs) != cudaSuccess)
                    rc = NVD_ERR_CUDA;
                if (rc == NVD_OK) rc = run_persistent(U, c, a, o.mode, KT, xdt, cs);
                if (rc == NVD_OK &&
                    cudaMemcpyAsync(u->h_res, w.res, (size_t)G * KT * sizeof(ColResult), cudaMemcpyDeviceToHost, cs) !=
                        cudaSuccess)
                    rc = NVD_ERR_CUDA;
                const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
                if (rc != NVD_OK || ec != cudaSuccess) {
                    if (graph) cudaGraphDestroy(graph);
                    cudaGetLastError();
                    u->graphs.erase(key);
                    if (rc == NVD_OK) {
                        set_error("nvd_ge_distance_batched: graph capture failed: %s", cudaGetErrorString(ec));
                        rc = NVD_ERR_CUDA;
                    }
                    return rc;
                }
                const cudaError_t ei = cudaGraphInstantiate(&cp->exec, graph, 0);
                cudaGraphDestroy(graph);
                if (ei != cudaSuccess) {
                    cudaGetLastError();
                    u->graphs.erase(key);
                    set_error("nvd_ge_distance_batched: graph instantiate failed: %s", cudaGetErrorString(ei));
                    return NVD_ERR_CUDA;
                }
                cap = std::move(cp);
            }
            NVD_TRY_CUDA(cudaGraphLaunch(cap->exec, cs));
            note_launch();
            NVD_TRY_CUDA(cudaEventRecord(u->ev_out, cs));
            NVD_TRY_CUDA(cudaStreamWaitEvent(s, u->ev_out, 0));
            NVD_TRY_CUDA(cudaStreamSynchronize(cs));
        }
        int err = 0;
        NVD_TRY_CUDA(cudaMemcpy(&err, c.err, 4, cudaMemcpyDeviceToHost));
        if (err) {
            set_error("nvd_ge_distance_batched: a bounded device wait gave up (status %d)", err);
            return err;
        }
        for (int i = 0; i < G; ++i) {
            const int kc = own[i].kc;
            for (int j = 0; j < kc; ++j) {
                const ColResult &r = u->h_res[(size_t)i * KT + j];
                const int64_t oi = out_off[i] + c0 + j;
                d2_out[oi] = r.d2;
                if (r.status != NVD_OK && overall != NVD_ERR_NUMERIC) overall = r.status;
                if (stats) {
                    stats[oi].iters = r.iters;
                    stats[oi].refine_steps = 0;
                    stats[oi].rel_resid = r.rr0 > 0.0 ? std::sqrt(std::max(r.rr, 0.0) / r.rr0) : 0.0;
                    stats[oi].status = r.status;
                    stats[oi].reserved = 0;
                }
            }
        }
    }
    if (overall != NVD_OK) set_error("nvd_ge_distance_batched: some pair ended with status %d", overall);
    return overall;
}

}  // namespace

extern "C" int nvd_ge_distance_batched(const nvd_graph_t *graphs, int32_t G, const int32_t *k_per,
                                       const void *const *x, const void *const *y, int32_t xdtype,
                                       const nvd_solve_opts *opts, double *d2_out, nvd_solve_stats *stats,
                                       nvd_stream_t stream) {
    clear_error();
    TraceRange trace("nvd_ge_distance_batched");
    try {
        return batched_impl(graphs, G, k_per, x, y, xdtype, opts, d2_out, stats, (cudaStream_t)stream);
    } catch (const std::bad_alloc &) {
        set_error("nvd_ge_distance_batched: host allocation failed");
        return NVD_ERR_OOM;
    } catch (...) {
        set_error("nvd_ge_distance_batched: unexpected host exception");
        return NVD_ERR_CUDA;
    }
}
