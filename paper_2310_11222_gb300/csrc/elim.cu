// Exact elimination of degree-1 and degree-2 nodes before the PCG solve (internal
// and C ABI: nvd_graph_eliminate, nvd_eliminate_host, NVD_SOLVE_ELIMINATE).
//
// Gaussian elimination of one node v of a graph Laplacian L leaves the Schur
// complement L' = L_rest - l_v l_v^T / d_v, again a graph Laplacian with no fill
// when v has at most two neighbours: a leaf disappears with its edge, a node with
// neighbours a, c is replaced by one edge a-c of conductance w_a w_c / d_v (the
// series rule).  For a right-hand side b that is mean-zero on every component,
//     b^T L^+ b = b'^T L'^+ b' + b_v^2 / d_v,   b'_u = b_u + b_v w_vu / d_v,
// so the d^2 of the GE equation (Section 3.1) on the whole graph is the reduced
// graph's d^2 of b' plus one term per eliminated node, and the PCG solve of
// Section 3.2 runs on the reduced graph only.  Sparse graphs (mean degree < 4,
// tree-like parts, long chains), where Jacobi PCG needs the most iterations, are
// the ones that shrink most.
//
// Nodes are eliminated in rounds.  The nodes of one round form an independent set
// (no two adjacent) and their neighbours are not eliminated in that round, so every
// b_v of a round is final when the round starts: the forward pass over a right-hand
// side is one parallel step per round, each record gathering the contributions of
// earlier records in a fixed order (no atomics; the result does not depend on
// scheduling).  A chain of length L goes in about log2(L) rounds.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "dispatch.h"
#include "solver.cuh"

namespace nvd {

// Host elimination of degree <= 2 nodes; records in round order.
struct ElimResult {
    std::vector<int32_t> rec_v;          // eliminated node of each record
    std::vector<double> rec_d;           // its weighted degree when eliminated
    std::vector<int32_t> rec_t0, rec_t1; // its neighbours then (-1: none), for the back-substitution
    std::vector<double> rec_f0, rec_f1;  // w_vt / d_v
    std::vector<int64_t> round_ptr;      // records of round t: [round_ptr[t], round_ptr[t+1])
    std::vector<int32_t> keep;           // kept nodes, increasing id
    std::vector<int64_t> red_rowptr;     // reduced graph on the indices of `keep`
    std::vector<int32_t> red_col;
    std::vector<double> red_w;
    // gather lists: b of record r = b_v + sum f * b(src); kept node i likewise
    std::vector<int64_t> rin_ptr, kin_ptr;
    std::vector<int32_t> rin_src, kin_src;
    std::vector<double> rin_f, kin_f;
};

static int eliminate_low_degree(int64_t n, const int64_t *rowptr, const int32_t *col, const double *w,
                                ElimResult *out) {
    struct E {
        int32_t u;
        double w;
    };
    std::vector<std::vector<E>> adj(n);
    for (int64_t v = 0; v < n; ++v)
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e)
            if (col[e] != v && w[e] != 0.0) adj[v].push_back({col[e], w[e]});
    std::vector<char> alive(n, 1);
    std::vector<int32_t> taken(n, -1), blocked(n, -1), rec_of(n, -1);
    std::vector<int32_t> &t0 = out->rec_t0, &t1 = out->rec_t1;
    std::vector<double> &f0 = out->rec_f0, &f1 = out->rec_f1;
    // distinct live neighbours of v with their summed conductances (parallel entries
    // added); returns their number, or 3 for "more than two".  Entries of eliminated
    // nodes are dropped from the list on the way.
    auto neighbours = [&](int32_t v, E *nb) {
        std::vector<E> &L = adj[v];
        size_t wr = 0;
        int m = 0;
        for (size_t q = 0; q < L.size(); ++q) {
            const E x = L[q];
            if (!alive[x.u]) continue;
            L[wr++] = x;
            if (m > 2) continue;
            int t = 0;
            while (t < m && nb[t].u != x.u) ++t;
            if (t == m) {
                if (m == 2) {
                    m = 3;
                    continue;
                }
                nb[m++] = {x.u, 0.0};
            }
            nb[t].w += x.w;
        }
        L.resize(wr);
        return m;
    };
    std::vector<int32_t> cur;
    for (int64_t v = 0; v < n; ++v) {
        E nb[2];
        const int m = neighbours((int32_t)v, nb);
        if (m >= 1 && m <= 2) cur.push_back((int32_t)v);
    }
    out->round_ptr.assign(1, 0);
    for (int32_t round = 0; !cur.empty(); ++round) {
        std::vector<int32_t> S;
        std::vector<E> snb;
        std::vector<int> sm;
        for (int32_t v : cur) {
            if (!alive[v] || taken[v] == round || blocked[v] == round) continue;
            E nb[2];
            const int m = neighbours(v, nb);
            if (m == 0 || m > 2) continue;
            bool free = true;
            for (int q = 0; q < m; ++q) free = free && taken[nb[q].u] != round;
            if (!free) continue;
            taken[v] = round;
            for (int q = 0; q < m; ++q) blocked[nb[q].u] = round;
            S.push_back(v);
            sm.push_back(m);
            for (int q = 0; q < 2; ++q) snb.push_back(q < m ? nb[q] : E{-1, 0.0});
        }
        if (S.empty()) break;
        std::vector<int32_t> next;
        for (size_t s = 0; s < S.size(); ++s) {
            const int32_t v = S[s];
            const E *nb = &snb[2 * s];
            const int m = sm[s];
            const double dv = nb[0].w + (m == 2 ? nb[1].w : 0.0);
            rec_of[v] = (int32_t)out->rec_v.size();
            out->rec_v.push_back(v);
            out->rec_d.push_back(dv);
            t0.push_back(nb[0].u);
            f0.push_back(nb[0].w / dv);
            t1.push_back(m == 2 ? nb[1].u : -1);
            f1.push_back(m == 2 ? nb[1].w / dv : 0.0);
            alive[v] = 0;
            if (m == 2) {
                const double wn = nb[0].w * nb[1].w / dv;
                adj[nb[0].u].push_back({nb[1].u, wn});
                adj[nb[1].u].push_back({nb[0].u, wn});
            }
            for (int q = 0; q < m; ++q) next.push_back(nb[q].u);
        }
        // the neighbours of this round's nodes and the candidates left over are
        // the next round's candidates (checked by their distinct live neighbours)
        for (int32_t v : cur)
            if (alive[v] && taken[v] != round) next.push_back(v);
        std::sort(next.begin(), next.end());
        next.erase(std::unique(next.begin(), next.end()), next.end());
        cur.clear();
        for (int32_t v : next) {
            if (!alive[v]) continue;
            E nb[2];
            const int m = neighbours(v, nb);
            if (m >= 1 && m <= 2) cur.push_back(v);
        }
        out->round_ptr.push_back((int64_t)out->rec_v.size());
    }
    // reduced graph on the kept nodes (parallel entries merged).  Rows a and c hold
    // the same multiset of conductances for their pair (every entry was added to
    // both rows), so sorting by (neighbour, conductance) and adding in that order
    // gives bitwise equal w_ac and w_ca: the reduced Laplacian is exactly symmetric.
    std::vector<int32_t> kidx(n, -1);
    for (int64_t v = 0; v < n; ++v)
        if (alive[v]) {
            kidx[v] = (int32_t)out->keep.size();
            out->keep.push_back((int32_t)v);
        }
    out->red_rowptr.assign(1, 0);
    std::vector<E> row;
    for (int32_t v : out->keep) {
        row.clear();
        for (const E &x : adj[v])
            if (alive[x.u] && x.u != v) row.push_back({kidx[x.u], x.w});
        std::sort(row.begin(), row.end(),
                  [](const E &a, const E &b) { return a.u < b.u || (a.u == b.u && a.w < b.w); });
        for (size_t q = 0; q < row.size(); ++q) {
            if (q > 0 && row[q].u == row[q - 1].u) {
                out->red_w.back() += row[q].w;
                continue;
            }
            out->red_col.push_back(row[q].u);
            out->red_w.push_back(row[q].w);
        }
        out->red_rowptr.push_back((int64_t)out->red_col.size());
    }
    // gather lists in record order
    const int64_t R = (int64_t)out->rec_v.size(), K = (int64_t)out->keep.size();
    std::vector<int64_t> rc(R + 1, 0), kc(K + 1, 0);
    for (int64_t r = 0; r < R; ++r)
        for (int32_t t : {t0[r], t1[r]}) {
            if (t < 0) continue;
            if (alive[t]) ++kc[kidx[t] + 1];
            else ++rc[rec_of[t] + 1];
        }
    for (int64_t i = 0; i < R; ++i) rc[i + 1] += rc[i];
    for (int64_t i = 0; i < K; ++i) kc[i + 1] += kc[i];
    out->rin_ptr = rc;
    out->kin_ptr = kc;
    out->rin_src.resize(rc[R]);
    out->rin_f.resize(rc[R]);
    out->kin_src.resize(kc[K]);
    out->kin_f.resize(kc[K]);
    for (int64_t r = 0; r < R; ++r)
        for (int q = 0; q < 2; ++q) {
            const int32_t t = q ? t1[r] : t0[r];
            const double f = q ? f1[r] : f0[r];
            if (t < 0) continue;
            if (alive[t]) {
                const int64_t pos = kc[kidx[t]]++;
                out->kin_src[pos] = (int32_t)r;
                out->kin_f[pos] = f;
            } else {
                const int64_t pos = rc[rec_of[t]]++;
                out->rin_src[pos] = (int32_t)r;
                out->rin_f[pos] = f;
            }
        }
    return NVD_OK;
}

struct ElimState {
    nvd_graph_t red = nullptr;           // the reduced graph
    int64_t n_rec = 0, n_keep = 0, red_nnz = 0;
    std::vector<int64_t> round_ptr;
    DevBuf rec_v, rec_d, rin_ptr, rin_src, rin_f, keep, kin_ptr, kin_src, kin_f, rec_t0, rec_t1, rec_f0, rec_f1;
    ~ElimState() {
        if (red) nvd_graph_destroy(red);
    }
};

void elim_state_delete(ElimState *e) { delete e; }

template <class T>
static int upload_vec(DevBuf &b, const std::vector<T> &v, cudaStream_t s) {
    NVD_TRY(b.alloc(std::max<size_t>(v.size(), 1) * sizeof(T)));
    if (!v.empty()) NVD_TRY_CUDA(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return NVD_OK;
}

// ------------------------------------------------------------------ kernels

// b of the records of one round: b_v + sum over earlier records of f * b(src).
__global__ void k_elim_round(int64_t r0, int64_t r1, const int32_t *__restrict__ rec_v,
                             const int64_t *__restrict__ rin_ptr, const int32_t *__restrict__ rin_src,
                             const double *__restrict__ rin_f, const double *__restrict__ delta,
                             double *__restrict__ rb) {
    for (int64_t r = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < r1;
         r += (int64_t)gridDim.x * blockDim.x) {
        double b = delta[rec_v[r]];
        for (int64_t e = rin_ptr[r]; e < rin_ptr[r + 1]; ++e) b += rin_f[e] * rb[rin_src[e]];
        rb[r] = b;
    }
}

// Reduced right-hand side of the kept nodes (the reduced graph's node order).
__global__ void k_elim_keep(int64_t K, const int32_t *__restrict__ keep, const int64_t *__restrict__ kin_ptr,
                            const int32_t *__restrict__ kin_src, const double *__restrict__ kin_f,
                            const double *__restrict__ delta, const double *__restrict__ rb,
                            double *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
        double b = delta[keep[i]];
        for (int64_t e = kin_ptr[i]; e < kin_ptr[i + 1]; ++e) b += kin_f[e] * rb[kin_src[e]];
        out[i] = b;
    }
}

// sum_r b_r^2 / d_r: per-block partials in a fixed order, then one block adds them
// in block order.
constexpr int EL_NT = 256;
__device__ __forceinline__ double el_block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = EL_NT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    return sh[0];
}
__global__ void k_elim_extra_part(int64_t R, const double *__restrict__ rb, const double *__restrict__ rec_d,
                                  double *__restrict__ part) {
    __shared__ double sh[EL_NT];
    double acc = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * EL_NT + threadIdx.x; r < R; r += (int64_t)gridDim.x * EL_NT)
        acc += rb[r] * rb[r] / rec_d[r];
    const double t = el_block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}
__global__ void k_elim_extra_final(int nb, const double *__restrict__ part, double *__restrict__ out) {
    __shared__ double sh[EL_NT];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += EL_NT) acc += part[b];
    const double t = el_block_sum(acc, sh);
    if (threadIdx.x == 0) *out = t;
}

// Back-substitution of one round (rounds in reverse order): an eliminated node's
// solution from its right-hand side and its neighbours at elimination time,
//     z_v = b_v / d_v + f_0 z_{t0} + f_1 z_{t1}   (f = w_vt / d_v),
// whose solutions are known (kept, or eliminated in a later round).
__global__ void k_elim_back(int64_t r0, int64_t r1, const int32_t *__restrict__ rec_v,
                            const double *__restrict__ rec_d, const int32_t *__restrict__ t0,
                            const int32_t *__restrict__ t1, const double *__restrict__ f0,
                            const double *__restrict__ f1, const double *__restrict__ rb, double *__restrict__ z) {
    for (int64_t r = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < r1;
         r += (int64_t)gridDim.x * blockDim.x) {
        double v = rb[r] / rec_d[r] + f0[r] * z[t0[r]];
        if (t1[r] >= 0) v += f1[r] * z[t1[r]];
        z[rec_v[r]] = v;
    }
}

// z[keep[i]] = the reduced graph's solution at its node i.
__global__ void k_elim_put_keep(int64_t K, const int32_t *__restrict__ keep, const double *__restrict__ zr,
                                double *__restrict__ z) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x)
        z[keep[i]] = zr[i];
}

// d2 = d2 of the reduced graph + the eliminated nodes' terms.
__global__ void k_elim_add(int32_t k, const double *__restrict__ a, const double *__restrict__ b,
                           double *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) out[j] = a[j] + b[j];
}

// ------------------------------------------------------------------ host

static int build_state(nvd_graph_s *g, cudaStream_t s) {
    std::vector<int32_t> col(g->nnz);
    std::vector<double> w(g->nnz);
    if (g->nnz) {
        NVD_TRY_CUDA(cudaMemcpyAsync(col.data(), g->colidx.p, g->nnz * 4, cudaMemcpyDeviceToHost, s));
        if (g->wdtype == NVD_F64) {
            NVD_TRY_CUDA(cudaMemcpyAsync(w.data(), g->w.p, g->nnz * 8, cudaMemcpyDeviceToHost, s));
            NVD_TRY_CUDA(cudaStreamSynchronize(s));
        } else {
            std::vector<float> wf(g->nnz);
            NVD_TRY_CUDA(cudaMemcpyAsync(wf.data(), g->w.p, g->nnz * 4, cudaMemcpyDeviceToHost, s));
            NVD_TRY_CUDA(cudaStreamSynchronize(s));
            for (int64_t i = 0; i < g->nnz; ++i) w[i] = wf[i];
        }
    }
    ElimResult er;
    NVD_TRY(eliminate_low_degree(g->n, g->h_rowptr.data(), col.data(), w.data(), &er));
    std::unique_ptr<ElimState, void (*)(ElimState *)> st(new ElimState(), elim_state_delete);
    st->n_rec = (int64_t)er.rec_v.size();
    st->n_keep = (int64_t)er.keep.size();
    st->red_nnz = (int64_t)er.red_col.size();
    st->round_ptr = er.round_ptr;
    NVD_TRY(upload_vec(st->rec_v, er.rec_v, s));
    NVD_TRY(upload_vec(st->rec_d, er.rec_d, s));
    NVD_TRY(upload_vec(st->rin_ptr, er.rin_ptr, s));
    NVD_TRY(upload_vec(st->rin_src, er.rin_src, s));
    NVD_TRY(upload_vec(st->rin_f, er.rin_f, s));
    NVD_TRY(upload_vec(st->keep, er.keep, s));
    NVD_TRY(upload_vec(st->kin_ptr, er.kin_ptr, s));
    NVD_TRY(upload_vec(st->kin_src, er.kin_src, s));
    NVD_TRY(upload_vec(st->kin_f, er.kin_f, s));
    NVD_TRY(upload_vec(st->rec_t0, er.rec_t0, s));
    NVD_TRY(upload_vec(st->rec_t1, er.rec_t1, s));
    NVD_TRY(upload_vec(st->rec_f0, er.rec_f0, s));
    NVD_TRY(upload_vec(st->rec_f1, er.rec_f1, s));
    NVD_TRY_CUDA(cudaStreamSynchronize(s));
    // the reduced graph: nodes = kept nodes of g's internal order (still
    // component-contiguous), bitwise symmetric by construction (parallel entries
    // merged in a fixed order both rows share); none when no edge is left
    // (every component went down to one node: d^2 is the eliminated terms alone)
    if (st->red_nnz > 0)
        NVD_TRY(nvd_graph_create(&st->red, st->n_keep, st->red_nnz, er.red_rowptr.data(), er.red_col.data(),
                                 er.red_w.data(), NVD_F64, NVD_GRAPH_SKIP_SYM_CHECK, (nvd_stream_t)s));
    g->elim = std::move(st);
    return NVD_OK;
}

int elim_distance(nvd_graph_t g, int32_t k, const void *x, const void *y, int32_t xdt,
                  const nvd_solve_opts *opts, double *d2_out, void *z_out, nvd_solve_stats *stats,
                  cudaStream_t s, bool idx) {
    if (!g || k < 0 || (xdt != NVD_F32 && xdt != NVD_F64)) {
        set_error("nvd_ge_distance: invalid argument");
        return NVD_ERR_INVALID_ARG;
    }
    if (k == 0) return NVD_OK;
    nvd_solve_opts o = *opts;
    if (!g->elim) {
        set_error("nvd_ge_distance: NVD_SOLVE_ELIMINATE needs nvd_graph_eliminate on the handle first");
        return NVD_ERR_INVALID_ARG;
    }
    if (!x || !y || !d2_out || (o.flags & NVD_SOLVE_HOST_INPUTS)) {
        set_error("nvd_ge_distance: NVD_SOLVE_ELIMINATE takes device x, y and needs d2_out");
        return NVD_ERR_INVALID_ARG;
    }
    TraceRange trace("nvd_ge_distance (eliminated)");
    ElimState &E = *g->elim;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != g->device) cudaSetDevice(g->device);
    struct Back {
        int prev, dev;
        ~Back() {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } back{cur, g->device};
    // projected delta of each pair in the internal layout (one column at a time)
    Plan *pl = nullptr;
    NVD_TRY(get_plan(g, 1, 8, 8, &pl));
    Ctx c;
    memset(&c, 0, sizeof(c));
    fill_graph_ctx(g, pl, &c);
    SolveWs w;
    NVD_TRY(setup_ws(g, pl, 1, 8, false, 1, &c, &w, s));
    int st = NVD_OK;
    const int64_t K = E.n_keep, R = E.n_rec;
    const int nbx = (int)std::max<int64_t>(1, std::min<int64_t>((R + EL_NT * 8 - 1) / (EL_NT * 8), 1024));
    double *bred = (double *)g->wsp("elim_b", (size_t)k * K * 8, &st);
    double *zero = (double *)g->wsp("elim_zero", (size_t)k * K * 8, &st);
    // the records' right-hand sides of every pair stay for the back-substitution
    // when z_out is asked for; otherwise one pair's at a time
    const int64_t rbs = std::max<int64_t>(R, 1);
    double *rb_all = (double *)g->wsp("elim_rb", (size_t)rbs * (z_out ? k : 1) * 8, &st);
    double *ex = (double *)g->wsp("elim_extra", (size_t)(3 * k + nbx) * 8, &st);
    double *zred = z_out ? (double *)g->wsp("elim_zred", (size_t)k * K * 8, &st) : nullptr;
    if (st) return st;
    double *d2r = ex + k, *d2f = ex + 2 * k, *part = ex + 3 * k;
    NVD_TRY_CUDA(cudaMemsetAsync(zero, 0, (size_t)k * K * 8, s));
    const size_t xsz = xdt == NVD_F64 ? 8 : 4;
    // pair j's inputs: [n] vectors of the x type, or (idx) one int32 node id each
    auto px = [&](const void *p, int32_t j) -> const void * {
        return idx ? (const void *)((const int32_t *)p + j) : (const void *)((const char *)p + (size_t)j * g->n * xsz);
    };
    for (int32_t j = 0; j < k; ++j) {
        double *rb = rb_all + (z_out ? (size_t)j * rbs : 0);
        c.own0 = Owner{px(x, j), px(y, j), nullptr, 0, g->n, 1, 0, g->nseg, idx ? 1 : 0};
        c.owners = nullptr;
        c.n_owner = 1;
        NVD_TRY_CUDA(cudaMemsetAsync(w.delta, 0, (size_t)g->n * 8, s));
        NVD_TRY_CUDA(cudaMemsetAsync(c.n_active, 0, 4, s));
        if (xdt == NVD_F64) {
            dev::OpFormDelta<double, 1> fd;
            fd.delta = w.delta;
            fd.fin.KT = 1;
            NVD_TRY((launch_vec<double, 1>(c, fd, s)));
        } else {
            dev::OpFormDelta<float, 1> fd;
            fd.delta = w.delta;
            fd.fin.KT = 1;
            NVD_TRY((launch_vec<double, 1>(c, fd, s)));
        }
        dev::OpInit<double, 1> oi;
        oi.src = w.delta; oi.writeback = w.delta;
        oi.x = (double *)w.x; oi.r = (double *)w.r; oi.p = (double *)w.p;
        oi.fin.KT = 1;
        NVD_TRY((launch_vec<double, 1>(c, oi, s)));
        for (size_t t = 0; t + 1 < E.round_ptr.size(); ++t) {
            const int64_t r0 = E.round_ptr[t], r1 = E.round_ptr[t + 1];
            if (r1 <= r0) continue;
            k_elim_round<<<(int)std::min<int64_t>((r1 - r0 + 255) / 256, 4096), 256, 0, s>>>(
                r0, r1, E.rec_v.as<int32_t>(), E.rin_ptr.as<int64_t>(), E.rin_src.as<int32_t>(),
                E.rin_f.as<double>(), w.delta, rb);
            note_launch();
            NVD_TRY_CUDA(cudaGetLastError());
        }
        k_elim_keep<<<(int)std::min<int64_t>((K + 255) / 256, 4096), 256, 0, s>>>(
            K, E.keep.as<int32_t>(), E.kin_ptr.as<int64_t>(), E.kin_src.as<int32_t>(), E.kin_f.as<double>(),
            w.delta, rb, bred + (size_t)j * K);
        note_launch();
        NVD_TRY_CUDA(cudaGetLastError());
        if (R > 0) {
            k_elim_extra_part<<<nbx, EL_NT, 0, s>>>(R, rb, E.rec_d.as<double>(), part);
            note_launch();
            k_elim_extra_final<<<1, EL_NT, 0, s>>>(nbx, part, ex + j);
            note_launch();
            NVD_TRY_CUDA(cudaGetLastError());
        } else {
            NVD_TRY_CUDA(cudaMemsetAsync(ex + j, 0, 8, s));
        }
    }
    // PCG on the reduced graph (all pairs), then add the eliminated nodes' terms
    nvd_solve_opts o2 = o;
    o2.flags = (o.flags & ~(NVD_SOLVE_ELIMINATE | NVD_SOLVE_HOST_INPUTS | NVD_SOLVE_NO_SYNC)) | NVD_SOLVE_D2_DEVICE;
    int rc = NVD_OK;
    if (E.red) {
        rc = nvd_ge_distance(E.red, k, bred, zero, NVD_F64, &o2, d2r, zred, stats, (nvd_stream_t)s);
        if (rc != NVD_OK && rc != NVD_ERR_NOT_CONVERGED && rc != NVD_ERR_NUMERIC) return rc;
    } else {
        // every component was eliminated down to one node: nothing left to solve
        NVD_TRY_CUDA(cudaMemsetAsync(d2r, 0, (size_t)k * 8, s));
        if (zred) NVD_TRY_CUDA(cudaMemsetAsync(zred, 0, (size_t)k * K * 8, s));
        if (stats)
            for (int32_t j = 0; j < k; ++j) stats[j] = nvd_solve_stats{0, 0, 0.0, NVD_OK, 0};
    }
    if (z_out) {
        // z of the full graph: the reduced solution on the kept nodes, the eliminated
        // nodes by back-substitution (last round first), then mean-zero per
        // component (OpFinal's means, OpZout's projection into the user layout)
        double *zf = (double *)w.x;
        for (int32_t j = 0; j < k; ++j) {
            const double *rb = rb_all + (size_t)j * rbs;
            NVD_TRY_CUDA(cudaMemsetAsync(zf, 0, (size_t)g->n * 8, s));
            k_elim_put_keep<<<(int)std::min<int64_t>((K + 255) / 256, 4096), 256, 0, s>>>(
                K, E.keep.as<int32_t>(), zred + (size_t)j * K, zf);
            note_launch();
            for (size_t t = E.round_ptr.size() - 1; t-- > 0;) {
                const int64_t r0 = E.round_ptr[t], r1 = E.round_ptr[t + 1];
                if (r1 <= r0) continue;
                k_elim_back<<<(int)std::min<int64_t>((r1 - r0 + 255) / 256, 4096), 256, 0, s>>>(
                    r0, r1, E.rec_v.as<int32_t>(), E.rec_d.as<double>(), E.rec_t0.as<int32_t>(),
                    E.rec_t1.as<int32_t>(), E.rec_f0.as<double>(), E.rec_f1.as<double>(), rb, zf);
                note_launch();
            }
            NVD_TRY_CUDA(cudaGetLastError());
            c.own0 = Owner{px(x, j), px(y, j), (char *)z_out + (size_t)j * g->n * xsz, 0, g->n, 1, 0, g->nseg,
                           idx ? 1 : 0};
            if (g->n_singleton > 0)
                NVD_TRY_CUDA(cudaMemsetAsync((char *)z_out + (size_t)j * g->n * xsz, 0, (size_t)g->n * xsz, s));
            dev::OpFinal<double, 1> of;
            of.x = zf; of.delta = w.delta;
            of.fin.KT = 1; of.fin.set_d2 = false;
            NVD_TRY((launch_vec<double, 1>(c, of, s)));
            if (xdt == NVD_F64) {
                dev::OpZout<double, double, 1> oz;
                oz.src = zf; oz.meanv = c.meanx;
                NVD_TRY((launch_vec<double, 1>(c, oz, s)));
            } else {
                dev::OpZout<double, float, 1> oz;
                oz.src = zf; oz.meanv = c.meanx;
                NVD_TRY((launch_vec<double, 1>(c, oz, s)));
            }
        }
    }
    const bool d2_dev = o.flags & NVD_SOLVE_D2_DEVICE;
    k_elim_add<<<(k + 127) / 128, 128, 0, s>>>(k, d2r, ex, d2_dev ? d2_out : d2f);
    note_launch();
    NVD_TRY_CUDA(cudaGetLastError());
    if (!d2_dev) NVD_TRY_CUDA(cudaMemcpyAsync(d2_out, d2f, (size_t)k * 8, cudaMemcpyDeviceToHost, s));
    NVD_TRY_CUDA(cudaStreamSynchronize(s));
    if (rc != NVD_OK) set_error("nvd_ge_distance: some pair ended with status %d (%s)", rc, nvd_status_string(rc));
    return rc;
}

}  // namespace nvd

using namespace nvd;

extern "C" int nvd_graph_eliminate(nvd_graph_t g, nvd_elim_info *info, nvd_stream_t stream) {
    clear_error();
    if (!g) {
        set_error("nvd_graph_eliminate: NULL handle");
        return NVD_ERR_INVALID_ARG;
    }
    try {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != g->device) cudaSetDevice(g->device);
        TraceRange trace("nvd_graph_eliminate");
        const int rc = build_state(g, (cudaStream_t)stream);
        if (cur >= 0 && cur != g->device) cudaSetDevice(cur);
        if (rc != NVD_OK) return rc;
        if (info) {
            info->n_kept = g->elim->n_keep;
            info->n_eliminated = g->elim->n_rec;
            info->rounds = (int32_t)g->elim->round_ptr.size() - 1;
            info->nnz_kept = g->elim->red_nnz;
        }
        return NVD_OK;
    } catch (const std::bad_alloc &) {
        set_error("nvd_graph_eliminate: host allocation failed");
        return NVD_ERR_OOM;
    } catch (...) {
        set_error("nvd_graph_eliminate: unexpected host exception");
        return NVD_ERR_CUDA;
    }
}

extern "C" int nvd_eliminate_host(int64_t n, const int64_t *rowptr, const int32_t *colidx, const double *w,
                                  int64_t *n_kept, int32_t *keep, int64_t *red_rowptr, int32_t *red_colidx,
                                  double *red_w, int32_t *rounds) {
    clear_error();
    if (n < 1 || !rowptr || !n_kept || (rowptr[n] > 0 && (!colidx || !w))) {
        set_error("nvd_eliminate_host: invalid argument");
        return NVD_ERR_INVALID_ARG;
    }
    try {
        ElimResult er;
        NVD_TRY(eliminate_low_degree(n, rowptr, colidx, w, &er));
        *n_kept = (int64_t)er.keep.size();
        if (rounds) *rounds = (int32_t)er.round_ptr.size() - 1;
        if (keep) std::copy(er.keep.begin(), er.keep.end(), keep);
        if (red_rowptr) std::copy(er.red_rowptr.begin(), er.red_rowptr.end(), red_rowptr);
        if (red_colidx) std::copy(er.red_col.begin(), er.red_col.end(), red_colidx);
        if (red_w) std::copy(er.red_w.begin(), er.red_w.end(), red_w);
        return NVD_OK;
    } catch (const std::bad_alloc &) {
        set_error("nvd_eliminate_host: host allocation failed");
        return NVD_ERR_OOM;
    }
}

extern "C" int nvd_eliminate_host_program(int64_t n, const int64_t *rowptr, const int32_t *colidx,
                                          const double *w, int64_t *counts, int32_t *rec_v, double *rec_d,
                                          int64_t *round_ptr, int64_t *rin_ptr, int32_t *rin_src, double *rin_f,
                                          int32_t *keep, int64_t *kin_ptr, int32_t *kin_src, double *kin_f,
                                          int32_t *rec_t0, int32_t *rec_t1, double *rec_f0, double *rec_f1) {
    clear_error();
    if (n < 1 || !rowptr || !counts || (rowptr[n] > 0 && (!colidx || !w))) {
        set_error("nvd_eliminate_host_program: invalid argument");
        return NVD_ERR_INVALID_ARG;
    }
    try {
        ElimResult er;
        NVD_TRY(eliminate_low_degree(n, rowptr, colidx, w, &er));
        counts[0] = (int64_t)er.rec_v.size();
        counts[1] = (int64_t)er.keep.size();
        counts[2] = (int64_t)er.rin_src.size();
        counts[3] = (int64_t)er.kin_src.size();
        counts[4] = (int64_t)er.round_ptr.size() - 1;
        if (!rec_v || !rec_d || !round_ptr || !rin_ptr || !rin_src || !rin_f || !keep || !kin_ptr || !kin_src ||
            !kin_f || !rec_t0 || !rec_t1 || !rec_f0 || !rec_f1)
            return NVD_OK;
        std::copy(er.rec_t0.begin(), er.rec_t0.end(), rec_t0);
        std::copy(er.rec_t1.begin(), er.rec_t1.end(), rec_t1);
        std::copy(er.rec_f0.begin(), er.rec_f0.end(), rec_f0);
        std::copy(er.rec_f1.begin(), er.rec_f1.end(), rec_f1);
        std::copy(er.rec_v.begin(), er.rec_v.end(), rec_v);
        std::copy(er.rec_d.begin(), er.rec_d.end(), rec_d);
        std::copy(er.round_ptr.begin(), er.round_ptr.end(), round_ptr);
        std::copy(er.rin_ptr.begin(), er.rin_ptr.end(), rin_ptr);
        std::copy(er.rin_src.begin(), er.rin_src.end(), rin_src);
        std::copy(er.rin_f.begin(), er.rin_f.end(), rin_f);
        std::copy(er.keep.begin(), er.keep.end(), keep);
        std::copy(er.kin_ptr.begin(), er.kin_ptr.end(), kin_ptr);
        std::copy(er.kin_src.begin(), er.kin_src.end(), kin_src);
        std::copy(er.kin_f.begin(), er.kin_f.end(), kin_f);
        return NVD_OK;
    } catch (const std::bad_alloc &) {
        set_error("nvd_eliminate_host_program: host allocation failed");
        return NVD_ERR_OOM;
    }
}

