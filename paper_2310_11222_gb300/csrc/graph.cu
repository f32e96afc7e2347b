// Graph handles: CSR intake, validation, degrees, connected components, work plans.
//
// The operator is the graph Laplacian L = D - W of Section 3.1 (undirected,
// positive weights).  Creation checks the input, drops self-loops, merges
// repeated entries, computes the weighted degrees D (and D^-1 for the Jacobi
// preconditioner), finds the connected components (whose per-component
// constants span the null space of L) and, if a component is not a contiguous
// node range, relabels the nodes so that every component is one -- the solver
// then treats each component as an independent "segment".
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>

#include "graph.h"

namespace nvd {

// ------------------------------------------------------------------ errors

static thread_local char g_last_error[512] = {0};

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}
void clear_error() { g_last_error[0] = 0; }
const char *last_error() { return g_last_error; }

int DevBuf::alloc(size_t b) {
    release();
    cudaError_t e = cudaMalloc(&p, b ? b : 16);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        set_error("cudaMalloc(%zu) failed: %s", b, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? NVD_ERR_OOM : NVD_ERR_CUDA;
    }
    bytes = b;
    return NVD_OK;
}

// ------------------------------------------------------------------ kernels

// flags[0] column out of range, [1] unsorted or repeated column, [2] self-loop,
// [3] weight <= 0 / NaN / Inf.  One warp per row.
template <class TW>
__global__ void k_check_rows(int64_t n, const int64_t *__restrict__ rowptr,
                             const int32_t *__restrict__ colidx, const TW *__restrict__ w,
                             int *flags) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int f0 = 0, f1 = 0, f2 = 0, f3 = 0;
    for (int64_t u = warp; u < n; u += nw) {
        const int64_t a = rowptr[u], b = rowptr[u + 1];
        for (int64_t e = a + lane; e < b; e += 32) {
            const int32_t v = colidx[e];
            if (v < 0 || v >= n) f0 = 1;
            if (v == u) f2 = 1;
            if (e > a && colidx[e - 1] >= v) f1 = 1;
            if (w) {
                const double x = (double)w[e];
                if (!(x > 0.0) || !isfinite(x)) f3 = 1;
            }
        }
    }
    f0 = __any_sync(0xffffffffu, f0);
    f1 = __any_sync(0xffffffffu, f1);
    f2 = __any_sync(0xffffffffu, f2);
    f3 = __any_sync(0xffffffffu, f3);
    if (lane == 0) {
        if (f0) atomicOr(flags + 0, 1);
        if (f1) atomicOr(flags + 1, 1);
        if (f2) atomicOr(flags + 2, 1);
        if (f3) atomicOr(flags + 3, 1);
    }
}

// Symmetry: every entry (u, v, w) needs (v, u, w) with the identical weight.
// Columns are sorted and unique here; one warp per row, binary search in row v.
template <class TW>
__global__ void k_check_sym(int64_t n, const int64_t *__restrict__ rowptr,
                            const int32_t *__restrict__ colidx, const TW *__restrict__ w,
                            int *bad) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int f = 0;
    for (int64_t u = warp; u < n; u += nw) {
        const int64_t a = rowptr[u], b = rowptr[u + 1];
        for (int64_t e = a + lane; e < b; e += 32) {
            const int32_t v = colidx[e];
            int64_t lo = rowptr[v], hi = rowptr[v + 1];
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (colidx[mid] < u) lo = mid + 1; else hi = mid;
            }
            if (lo >= rowptr[v + 1] || colidx[lo] != u) f = 1;
            else if (w && w[lo] != w[e]) f = 1;
        }
    }
    if (__any_sync(0xffffffffu, f) && lane == 0) atomicOr(bad, 1);
}

// Weighted degree D_uu = sum_v w_uv (FP64, fixed lane-strided order + butterfly).
template <class TW>
__global__ void k_degree(int64_t n, const int64_t *__restrict__ rowptr, const TW *__restrict__ w,
                         double *deg64, double *dinv64, float *deg32, float *dinv32) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nw) {
        const int64_t a = rowptr[u], b = rowptr[u + 1];
        double s = 0.0;
        for (int64_t e = a + lane; e < b; e += 32) s += w ? (double)w[e] : 1.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) {
            deg64[u] = s;
            dinv64[u] = s > 0.0 ? 1.0 / s : 0.0;
            deg32[u] = (float)s;
            dinv32[u] = s > 0.0 ? (float)(1.0 / s) : 0.0f;
        }
    }
}

template <class T>
__global__ void k_fill(T *p, int64_t n, T v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_round_w32(const double *__restrict__ w, float *w32, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        w32[i] = (float)w[i];
}

// flag = 1 if some weight is <= 0, NaN or infinite.
template <class TW>
__global__ void k_check_weights(int64_t n, const TW *__restrict__ w, int *flag) {
    int f = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = (double)w[i];
        if (!(x > 0.0) || !isfinite(x)) f = 1;
    }
    if (__any_sync(0xffffffffu, f) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// New weights of the handle's entries from the caller's entries: internal entry e
// sums the user entries isrc[iptr[e] .. iptr[e+1]) in that (increasing) order in
// FP64, as the creation's cleaning merged repeated entries.
template <class TW>
__global__ void k_gather_weights(int64_t nnz, const int64_t *__restrict__ iptr, const int64_t *__restrict__ isrc,
                                 const TW *__restrict__ wu, TW *__restrict__ wi) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int64_t q = iptr[e]; q < iptr[e + 1]; ++q) t += (double)wu[isrc[q]];
        wi[e] = (TW)t;
    }
}

// Connected components by hooking and pointer jumping.  parent[] only ever
// decreases and always points to a smaller-or-equal node, so find() terminates;
// at the fixed point every node points at the smallest node of its component.
__device__ __forceinline__ int32_t cc_find(const int32_t *parent, int32_t x) {
    for (;;) {
        const int32_t p = __ldcg(parent + x);
        if (p == x) return x;
        x = p;
    }
}

__global__ void k_cc_hook(int64_t n, const int64_t *__restrict__ rowptr,
                          const int32_t *__restrict__ colidx, int32_t *parent, int *changed) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int ch = 0;
    for (int64_t u = warp; u < n; u += nw) {
        const int64_t a = rowptr[u], b = rowptr[u + 1];
        for (int64_t e = a + lane; e < b; e += 32) {
            const int32_t v = colidx[e];
            if (v == u) continue;
            const int32_t ru = cc_find(parent, (int32_t)u), rv = cc_find(parent, v);
            if (ru != rv) {
                const int32_t lo = ru < rv ? ru : rv, hi = ru < rv ? rv : ru;
                atomicMin(parent + hi, lo);
                ch = 1;
            }
        }
    }
    if (__any_sync(0xffffffffu, ch) && lane == 0) atomicOr(changed, 1);
}

__global__ void k_cc_compress(int64_t n, int32_t *parent) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        parent[i] = cc_find(parent, (int32_t)i);
}

static int grid_for(int64_t work, int threads_per_item, int num_sms) {
    int64_t b = (work * threads_per_item + 255) / 256;
    int64_t cap = (int64_t)num_sms * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

// ------------------------------------------------------------------ host helpers

namespace {

struct HostCSR {
    std::vector<int64_t> rowptr;
    std::vector<int32_t> col;
    std::vector<double> w;       // weights (as double; converted back to wdtype on upload)
    std::vector<int64_t> uent;   // user entry -> entry of this CSR (-1 dropped)
};

// Drop self-loops, sort each row by column, merge repeated columns (summing).
void clean_csr(int64_t n, const std::vector<int64_t> &rp, const std::vector<int32_t> &col,
               const std::vector<double> &w, HostCSR &out) {
    const int64_t nnz = rp[n];
    out.rowptr.assign(n + 1, 0);
    out.col.clear();
    out.w.clear();
    out.uent.assign(nnz, -1);
    std::vector<int64_t> idx;
    for (int64_t u = 0; u < n; ++u) {
        idx.clear();
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e)
            if (col[e] != u) idx.push_back(e);
        std::stable_sort(idx.begin(), idx.end(),
                         [&](int64_t a, int64_t b) { return col[a] < col[b]; });
        for (size_t t = 0; t < idx.size(); ++t) {
            const int64_t e = idx[t];
            if (t > 0 && col[idx[t - 1]] == col[e]) {
                out.w.back() += w[e];
            } else {
                out.col.push_back(col[e]);
                out.w.push_back(w[e]);
            }
            out.uent[e] = (int64_t)out.col.size() - 1;
        }
        out.rowptr[u + 1] = (int64_t)out.col.size();
    }
}

template <class T>
int upload_padded(nvd::DevBuf &buf, const T *host, int64_t n, cudaStream_t s) {
    const int64_t npad = ((n + 3) / 4) * 4 + 4;
    NVD_TRY(buf.alloc((size_t)npad * sizeof(T)));
    NVD_TRY_CUDA(cudaMemsetAsync(buf.p, 0, (size_t)npad * sizeof(T), s));
    if (n > 0)
        NVD_TRY_CUDA(cudaMemcpyAsync(buf.p, host, (size_t)n * sizeof(T), cudaMemcpyHostToDevice, s));
    return NVD_OK;
}

int upload_weights(nvd_graph_s *g, const std::vector<double> &w, cudaStream_t s) {
    if (g->wdtype == NVD_F64) return upload_padded(g->w, w.data(), (int64_t)w.size(), s);
    std::vector<float> wf(w.size());
    for (size_t i = 0; i < w.size(); ++i) wf[i] = (float)w[i];
    NVD_TRY(upload_padded(g->w, wf.data(), (int64_t)wf.size(), s));
    NVD_TRY_CUDA(cudaStreamSynchronize(s));
    return NVD_OK;
}

int download_csr(nvd_graph_s *g, std::vector<int32_t> &col, std::vector<double> &w, cudaStream_t s) {
    col.resize(g->nnz);
    w.resize(g->nnz);
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
    return NVD_OK;
}

template <class TW>
int run_checks(nvd_graph_s *g, bool have_w, int *flags_h, cudaStream_t s) {
    nvd::DevBuf flags;
    NVD_TRY(flags.alloc(4 * sizeof(int)));
    NVD_TRY_CUDA(cudaMemsetAsync(flags.p, 0, 4 * sizeof(int), s));
    k_check_rows<TW><<<nvd::grid_for(g->n, 32, g->num_sms), 256, 0, s>>>(
        g->n, g->rowptr.as<int64_t>(), g->colidx.as<int32_t>(),
        have_w ? g->w.as<TW>() : nullptr, flags.as<int>());
    NVD_TRY_CUDA(cudaGetLastError());
    NVD_TRY_CUDA(cudaMemcpyAsync(flags_h, flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    NVD_TRY_CUDA(cudaStreamSynchronize(s));
    return NVD_OK;
}

template <class TW>
int run_sym(nvd_graph_s *g, int *bad_h, cudaStream_t s, const TW *w = nullptr) {
    nvd::DevBuf bad;
    NVD_TRY(bad.alloc(sizeof(int)));
    NVD_TRY_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    k_check_sym<TW><<<nvd::grid_for(g->n, 32, g->num_sms), 256, 0, s>>>(
        g->n, g->rowptr.as<int64_t>(), g->colidx.as<int32_t>(), w ? w : g->w.as<TW>(), bad.as<int>());
    NVD_TRY_CUDA(cudaGetLastError());
    NVD_TRY_CUDA(cudaMemcpyAsync(bad_h, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    NVD_TRY_CUDA(cudaStreamSynchronize(s));
    return NVD_OK;
}

int run_degree(nvd_graph_s *g, cudaStream_t s) {
    const int64_t n = g->n;
    NVD_TRY(g->deg64.ensure(n * 8));
    NVD_TRY(g->dinv64.ensure(n * 8));
    NVD_TRY(g->deg32.ensure(n * 4));
    NVD_TRY(g->dinv32.ensure(n * 4));
    const int grid = nvd::grid_for(n, 32, g->num_sms);
    if (g->wdtype == NVD_F64)
        k_degree<double><<<grid, 256, 0, s>>>(n, g->rowptr.as<int64_t>(), g->w.as<double>(),
                                              g->deg64.as<double>(), g->dinv64.as<double>(),
                                              g->deg32.as<float>(), g->dinv32.as<float>());
    else
        k_degree<float><<<grid, 256, 0, s>>>(n, g->rowptr.as<int64_t>(), g->w.as<float>(),
                                             g->deg64.as<double>(), g->dinv64.as<double>(),
                                             g->deg32.as<float>(), g->dinv32.as<float>());
    NVD_TRY_CUDA(cudaGetLastError());
    return NVD_OK;
}

int run_components(nvd_graph_s *g, std::vector<int32_t> &root, cudaStream_t s) {
    const int64_t n = g->n;
    nvd::DevBuf parent, changed;
    NVD_TRY(parent.alloc(n * 4));
    NVD_TRY(changed.alloc(sizeof(int)));
    std::vector<int32_t> iota(n);
    std::iota(iota.begin(), iota.end(), 0);
    NVD_TRY_CUDA(cudaMemcpyAsync(parent.p, iota.data(), n * 4, cudaMemcpyHostToDevice, s));
    int h_changed = 1;
    const int grid = nvd::grid_for(n, 32, g->num_sms);
    int rounds = 0;
    for (; h_changed && rounds < 4096; ++rounds) {
        NVD_TRY_CUDA(cudaMemsetAsync(changed.p, 0, sizeof(int), s));
        k_cc_hook<<<grid, 256, 0, s>>>(n, g->rowptr.as<int64_t>(), g->colidx.as<int32_t>(),
                                       parent.as<int32_t>(), changed.as<int>());
        k_cc_compress<<<nvd::grid_for(n, 1, g->num_sms), 256, 0, s>>>(n, parent.as<int32_t>());
        NVD_TRY_CUDA(cudaGetLastError());
        NVD_TRY_CUDA(cudaMemcpyAsync(&h_changed, changed.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        NVD_TRY_CUDA(cudaStreamSynchronize(s));
    }
    if (h_changed) {
        set_error("connected components did not converge in %d rounds", rounds);
        return NVD_ERR_CUDA;
    }
    root.resize(n);
    NVD_TRY_CUDA(cudaMemcpyAsync(root.data(), parent.p, n * 4, cudaMemcpyDeviceToHost, s));
    NVD_TRY_CUDA(cudaStreamSynchronize(s));
    return NVD_OK;
}

}  // namespace

int target_blocks(const nvd_graph_s *g) { return 2 * g->num_sms * 8; }

// ------------------------------------------------------------------ TMA tensor maps

int tma_map(const void *base, int64_t rows, int kt, int szv, CUtensorMap *out) {
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::map<std::tuple<uintptr_t, int64_t, int, int>, CUtensorMap> cache;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple((uintptr_t)base, rows, kt, szv);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *out = it->second;
        return NVD_OK;
    }
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                               cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            set_error("TMA: cuTensorMapEncodeTiled is not available from the driver");
            return NVD_ERR_UNSUPPORTED;
        }
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    if (((uintptr_t)base & 15) || rows < 1 || rows > (int64_t)1 << 31 || (kt * szv) % 16 || kt > 256) {
        set_error("TMA: unsupported array for a tensor map (base %p, %lld rows of %d x %d bytes)", base,
                  (long long)rows, kt, szv);
        return NVD_ERR_UNSUPPORTED;
    }
    CUtensorMap m;
    const cuuint64_t dims[2] = {(cuuint64_t)kt, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kt * (cuuint64_t)szv};
    const cuuint32_t box[2] = {(cuuint32_t)kt, 1u};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = encode(&m, szv == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                              const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("TMA: cuTensorMapEncodeTiled failed (%d)", (int)r);
        return NVD_ERR_CUDA;
    }
    if (cache.size() > 256) cache.clear();
    cache[key] = m;
    *out = m;
    return NVD_OK;
}

// CTAs per SM of one vector pass: one column 4 (64 registers each), several
// columns 2 (128 registers each), i.e. one full wave either way.
#ifndef VEC_PER_SM
#define VEC_PER_SM(KT) ((KT) == 1 ? 4 : 2)
#endif

uint64_t next_graph_id() {
    static std::atomic<uint64_t> ctr{1};
    return ctr.fetch_add(1);
}

// ------------------------------------------------------------------ plans

// Fill the sliced copy of the light rows from the CSR: thread t is lane group r of
// slice t / H; entry j of its row goes to sl_base[slice] + j*H + r (consecutive
// threads write consecutive addresses).  Padding (rows shorter than the slice's
// longest, and empty lane groups) gets weight 0 on a column the row reads anyway
// (its own node; for an empty lane group the slice's first row).
template <class TWI, class TWO>
__global__ void k_fill_slices(int64_t n_slices, int H, const int64_t *__restrict__ sl_base,
                              const int32_t *__restrict__ sl_row, const int64_t *__restrict__ rowptr,
                              const int32_t *__restrict__ colidx, const TWI *__restrict__ w,
                              int32_t *__restrict__ sl_col, TWO *__restrict__ sl_w) {
    const int64_t nt = n_slices * H;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = t / H;
        const int r = (int)(t % H);
        const int64_t base = sl_base[sl];
        const int64_t L = (sl_base[sl + 1] - base) / H;
        const int32_t row = sl_row[t];
        const int32_t pad = row >= 0 ? row : sl_row[sl * H];
        const int64_t e0 = row >= 0 ? rowptr[row] : 0;
        const int64_t d = row >= 0 ? rowptr[row + 1] - e0 : 0;
        for (int64_t j = 0; j < L; ++j) {
            const bool in = j < d;
            sl_col[base + j * H + r] = in ? colidx[e0 + j] : pad;
            sl_w[base + j * H + r] = in ? (TWO)w[e0 + j] : (TWO)0;
        }
    }
}

// Light slices of a stream plan (stream.cuh): step 0 holds the slice's rows -- their own
// rows of the vector are gathered first -- with the rows' degrees as weights (-0
// marks an empty lane group, whose column is the slice's first row); steps 1..L the
// rows' entries, padded with zero weights on the row's own column; the weights of
// the last step are negated (sign bit set: the slice ends there, -0 for padding).
template <class TWI, class TA>
__global__ void k_fill_slices_tma(int64_t n_slices, int H, const int64_t *__restrict__ sl_base,
                                  const int32_t *__restrict__ sl_row, const int64_t *__restrict__ rowptr,
                                  const int32_t *__restrict__ colidx, const TWI *__restrict__ w,
                                  const TA *__restrict__ deg, int32_t *__restrict__ sl_col, TA *__restrict__ sl_w) {
    const int64_t nt = n_slices * H;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = t / H;
        const int r = (int)(t % H);
        const int64_t base = sl_base[sl];
        const int64_t L = (sl_base[sl + 1] - base) / H - 1;
        const int32_t row = sl_row[t];
        const int32_t own = row >= 0 ? row : sl_row[sl * H];
        sl_col[base + r] = own;
        sl_w[base + r] = row >= 0 ? deg[row] : -(TA)0;
        const int64_t e0 = row >= 0 ? rowptr[row] : 0;
        const int64_t d = row >= 0 ? rowptr[row + 1] - e0 : 0;
        for (int64_t j = 0; j < L; ++j) {
            const bool in = j < d;
            const TA wv = in ? (TA)w[e0 + j] : (TA)0;
            sl_col[base + (j + 1) * H + r] = in ? colidx[e0 + j] : own;
            sl_w[base + (j + 1) * H + r] = j == L - 1 ? -wv : wv;
        }
    }
}

// Heavy-row chunks of a stream plan as slices of their own (item.pad = the slice): entry
// j*H + g of the chunk at step j, lane group g (the CSR order), padded past the chunk
// with zero weights on the row's own column, the last step's weights negated.
template <class TWI, class TA>
__global__ void k_fill_chunks_tma(int64_t n_items, int H, const SpItem *__restrict__ items,
                                  const int64_t *__restrict__ sl_base, const int32_t *__restrict__ colidx,
                                  const TWI *__restrict__ w, int32_t *__restrict__ sl_col, TA *__restrict__ sl_w) {
    const int64_t nt = n_items * H;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt;
         t += (int64_t)gridDim.x * blockDim.x) {
        const SpItem it = items[t / H];
        const int r = (int)(t % H);
        const int64_t base = sl_base[it.pad];
        const int64_t S = (sl_base[it.pad + 1] - base) / H;
        for (int64_t j = 0; j < S; ++j) {
            const int64_t e = it.e0 + j * H + r;
            const bool in = e < it.e1;
            const TA wv = in ? (TA)w[e] : (TA)0;
            sl_col[base + j * H + r] = in ? colidx[e] : it.r0;
            sl_w[base + j * H + r] = j == S - 1 ? -wv : wv;
        }
    }
}

// (Re)write the sliced copy of a plan's light rows from the handle's CSR (after the
// plan is built, and after new weights).
static int fill_plan_slices(nvd_graph_s *g, Plan *pl, cudaStream_t s) {
    if (pl->n_slices == 0) return NVD_OK;
    const int H = sp_slice_rows(pl->KT, pl->szv);
    if (pl->stream) {
        // stream plans: weights in the solve's accumulator type (they carry the degrees)
        const int64_t *rpd = g->rowptr.as<int64_t>();
        const int32_t *cid = g->colidx.as<int32_t>();
        const int64_t *sb = pl->sl_base.as<int64_t>();
        const int32_t *sr = pl->sl_row.as<int32_t>();
        int32_t *sc = pl->sl_col.as<int32_t>();
        const SpItem *it = pl->items.as<SpItem>();
        const int gl = grid_for(std::max<int64_t>(pl->n_light_slices * H, 1), 1, g->num_sms);
        const int gh = grid_for(std::max<int64_t>(pl->n_items * H, 1), 1, g->num_sms);
        if (pl->szv == 8) {
            double *sw = pl->sl_w.as<double>();
            if (g->wdtype == NVD_F64) {
                if (pl->n_light_slices)
                    k_fill_slices_tma<double, double><<<gl, 256, 0, s>>>(pl->n_light_slices, H, sb, sr, rpd, cid,
                                                                         g->w.as<double>(), g->deg64.as<double>(), sc, sw);
                if (pl->n_items)
                    k_fill_chunks_tma<double, double><<<gh, 256, 0, s>>>(pl->n_items, H, it, sb, cid, g->w.as<double>(),
                                                                         sc, sw);
            } else {
                if (pl->n_light_slices)
                    k_fill_slices_tma<float, double><<<gl, 256, 0, s>>>(pl->n_light_slices, H, sb, sr, rpd, cid,
                                                                        g->w.as<float>(), g->deg64.as<double>(), sc, sw);
                if (pl->n_items)
                    k_fill_chunks_tma<float, double><<<gh, 256, 0, s>>>(pl->n_items, H, it, sb, cid, g->w.as<float>(),
                                                                        sc, sw);
            }
        } else {
            float *sw = pl->sl_w.as<float>();
            if (g->wdtype == NVD_F64) {
                if (pl->n_light_slices)
                    k_fill_slices_tma<double, float><<<gl, 256, 0, s>>>(pl->n_light_slices, H, sb, sr, rpd, cid,
                                                                        g->w.as<double>(), g->deg32.as<float>(), sc, sw);
                if (pl->n_items)
                    k_fill_chunks_tma<double, float><<<gh, 256, 0, s>>>(pl->n_items, H, it, sb, cid, g->w.as<double>(),
                                                                        sc, sw);
            } else {
                if (pl->n_light_slices)
                    k_fill_slices_tma<float, float><<<gl, 256, 0, s>>>(pl->n_light_slices, H, sb, sr, rpd, cid,
                                                                       g->w.as<float>(), g->deg32.as<float>(), sc, sw);
                if (pl->n_items)
                    k_fill_chunks_tma<float, float><<<gh, 256, 0, s>>>(pl->n_items, H, it, sb, cid, g->w.as<float>(),
                                                                       sc, sw);
            }
        }
        NVD_TRY_CUDA(cudaGetLastError());
        return NVD_OK;
    }
    const bool w64 = pl->szv == 8 && g->wdtype == NVD_F64;
    const int grid = grid_for(pl->n_slices * H, 1, g->num_sms);
    const int64_t *rpd = g->rowptr.as<int64_t>();
    const int32_t *cid = g->colidx.as<int32_t>();
    const int64_t *sb = pl->sl_base.as<int64_t>();
    const int32_t *sr = pl->sl_row.as<int32_t>();
    int32_t *sc = pl->sl_col.as<int32_t>();
    if (g->wdtype == NVD_F64 && w64)
        k_fill_slices<double, double><<<grid, 256, 0, s>>>(pl->n_slices, H, sb, sr, rpd, cid, g->w.as<double>(), sc,
                                                           pl->sl_w.as<double>());
    else if (g->wdtype == NVD_F64)
        k_fill_slices<double, float><<<grid, 256, 0, s>>>(pl->n_slices, H, sb, sr, rpd, cid, g->w.as<double>(), sc,
                                                          pl->sl_w.as<float>());
    else
        k_fill_slices<float, float><<<grid, 256, 0, s>>>(pl->n_slices, H, sb, sr, rpd, cid, g->w.as<float>(), sc,
                                                         pl->sl_w.as<float>());
    NVD_TRY_CUDA(cudaGetLastError());
    return NVD_OK;
}

int get_plan(nvd_graph_s *g, int KT, int szv, int sza, Plan **out, bool allow_stream) {
    // gather mode of this plan: 0 register slices, 1 register stream, 2 TMA stream,
    // 3 asynchronous-copy stream (2 and 3 for rows of 64 or 128 bytes)
    const int gm = (!allow_stream || KT == 1 || g->sp.gather <= 0) ? 0
                   : (g->sp.gather >= 2 && tma_tile(KT, szv)) ? std::min(g->sp.gather, 3) : 1;
    const bool tma = gm != 0;   // stream layout (the name of the TMA plans it began with)
    const int64_t key = ((int64_t)(KT * 256 + szv * 16 + sza) << 32) | ((int64_t)gm << 30) |
                        ((int64_t)g->sp.row_max_pct << 16) | (int64_t)g->sp.blocks_pct;
    auto it = g->plans.find(key);
    if (it != g->plans.end()) {
        *out = it->second.get();
        return NVD_OK;
    }
    std::unique_ptr<Plan> pl(new Plan());
    pl->KT = KT;
    pl->szv = szv;
    pl->sza = sza;
    pl->sp = g->sp;
    const int64_t RMAX = std::max<int64_t>(
        1, (int64_t)(tma ? sp_row_max_stream(KT, szv) : sp_row_max(KT, szv)) * g->sp.row_max_pct / 100);
    const int64_t LONG = sp_long_max(KT);
    const int64_t CH = tma ? sp_chunk_stream(KT, szv) : sp_chunk(KT, szv);
    const int H = sp_slice_rows(KT, szv);
    const std::vector<int64_t> &rp = g->h_rowptr;
    const int nseg = g->nseg;

    // heavy rows: a whole-row sub-item (KT = 1, up to LONG entries) or chunks of CH
    // entries; items are listed segment by segment
    std::vector<SpItem> items;
    std::vector<int32_t> seg_heavy_off(nseg + 1, 0);
    std::vector<int64_t> seg_item_off(nseg + 1, 0);
    int32_t nheavy = 0, nchunks = 0;
    double ltot = 0.0;
    for (int s = 0; s < nseg; ++s) {
        seg_item_off[s] = (int64_t)items.size();
        seg_heavy_off[s] = nheavy;
        for (int64_t r = g->h_seg_begin[s]; r < g->h_seg_end[s]; ++r) {
            const int64_t d = rp[r + 1] - rp[r];
            if (d <= RMAX) {
                ltot += (double)d + 1.0;
            } else if (d <= LONG) {
                SpItem si{};
                si.r0 = (int32_t)r;
                si.r1 = (int32_t)(r + 1);
                si.kind = 2;
                si.e0 = rp[r];
                si.e1 = rp[r + 1];
                items.push_back(si);
            } else {
                const int32_t nch = (int32_t)((d + CH - 1) / CH);
                for (int32_t q = 0; q < nch; ++q) {
                    SpItem si{};
                    si.r0 = (int32_t)r;
                    si.r1 = (int32_t)(r + 1);
                    si.kind = 1;
                    si.hrow = nheavy;
                    si.e0 = rp[r] + (int64_t)q * CH;
                    si.e1 = std::min(rp[r] + (int64_t)(q + 1) * CH, rp[r + 1]);
                    si.hbase = nchunks;
                    si.hchunk = q;
                    si.nchunk = nch;
                    items.push_back(si);
                }
                ++nheavy;
                nchunks += nch;
            }
        }
    }
    seg_item_off[nseg] = (int64_t)items.size();
    seg_heavy_off[nseg] = nheavy;

    // Light blocks: the light rows of a segment, in order, cut into blocks of whole
    // warp rounds (NWARP slices of H rows) of about `target` work (entries + rows);
    // inside a block the rows are sorted by length (longest first, ties by row) and
    // dealt into slices.  Heavy blocks follow their segment's light blocks.
    // (stream plans: half as many, larger light blocks; their warps split a block's
    // slices statically, which balances better on more work)
    const int T = std::max(1, (tma ? target_blocks(g) / 2 : target_blocks(g)) * g->sp.blocks_pct / 100);
    const double target = ltot / T;
    // block sizes in whole slices (warps take a block's slices as they free up)
    const int64_t QR = (int64_t)H;
    std::vector<Block> sblk;
    std::vector<int32_t> seg_sblk_off(nseg + 1, 0);
    std::vector<int64_t> sl_base(1, 0);
    std::vector<int32_t> sl_row;
    std::vector<int64_t> rows, lens;
    auto emit_block = [&](int s) {
        std::vector<int64_t> ord(rows.size());
        for (size_t q = 0; q < ord.size(); ++q) ord[q] = (int64_t)q;
        std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return lens[x] > lens[y]; });
        const int64_t first = (int64_t)sl_base.size() - 1;
        for (size_t q0 = 0; q0 < ord.size(); q0 += H) {
            int64_t L = 0;
            for (int r = 0; r < H; ++r) {
                const size_t q = q0 + r;
                sl_row.push_back(q < ord.size() ? (int32_t)rows[ord[q]] : -1);
                if (q < ord.size()) L = std::max(L, lens[ord[q]]);
            }
            // stream plans: one step more for the rows' own vector rows, at least one entry step
            sl_base.push_back(sl_base.back() + (tma ? std::max<int64_t>(L, 1) + 1 : L) * H);
        }
        sblk.push_back(Block{first, (int64_t)sl_base.size() - 1, s, 0, (int32_t)rows.front(),
                             (int32_t)(rows.back() - rows.front() + 1)});
        rows.clear();
        lens.clear();
    };
    // one column: a block's rows span at most sp_span_max() rows
    const int64_t SPAN = KT == 1 ? sp_span_max() : INT64_MAX;
    for (int s = 0; s < nseg; ++s) {
        seg_sblk_off[s] = (int32_t)sblk.size();
        double acc = 0.0;
        for (int64_t r = g->h_seg_begin[s]; r < g->h_seg_end[s]; ++r) {
            const int64_t d = rp[r + 1] - rp[r];
            if (d > RMAX) continue;
            if (!rows.empty() && r - rows.front() + 1 > SPAN) {
                emit_block(s);
                acc = 0.0;
            }
            rows.push_back(r);
            lens.push_back(d);
            acc += (double)d + 1.0;
            if ((int64_t)rows.size() % QR == 0 && acc >= target) {
                emit_block(s);
                acc = 0.0;
            }
        }
        if (!rows.empty()) emit_block(s);
        const size_t per = (KT == 1 || tma) ? (size_t)NWARP : 4;   // stream plans: one chunk per warp
        const int64_t h0 = seg_item_off[s], h1 = seg_item_off[s + 1];
        for (int64_t q = h0; q < h1; q += (int64_t)per)
            sblk.push_back(Block{q, std::min<int64_t>(h1, q + (int64_t)per), s, 1, 0, 0});
    }
    seg_sblk_off[nseg] = (int32_t)sblk.size();

    // Vector blocks: one wave of equal blocks, VEC_PER_SM(KT) per SM (the FP64 units
    // are per SM, so every SM gets the same share), at least 1024 row-columns each,
    // split over the segments in proportion to their rows.
    std::vector<Block> vblk;
    std::vector<int32_t> seg_vblk_off(nseg + 1, 0);
    int64_t rows_tot = 0;
    for (int s = 0; s < nseg; ++s) rows_tot += g->h_seg_end[s] - g->h_seg_begin[s];
    const int64_t TV = (int64_t)VEC_PER_SM(KT) * g->num_sms;
    for (int s = 0; s < nseg; ++s) {
        seg_vblk_off[s] = (int32_t)vblk.size();
        const int64_t a = g->h_seg_begin[s], b = g->h_seg_end[s], nr = b - a;
        int64_t nb = (int64_t)((double)TV * nr / (rows_tot > 0 ? rows_tot : 1) + 0.5);
        const int64_t maxb = std::max<int64_t>(1, (nr * KT + 1023) / 1024);
        nb = std::max<int64_t>(1, std::min<int64_t>(nb, maxb));
        for (int64_t k = 0; k < nb; ++k)
            vblk.push_back(Block{a + nr * k / nb, a + nr * (k + 1) / nb, s, 0, 0, 0});
    }
    seg_vblk_off[nseg] = (int32_t)vblk.size();

    // each warp of a light block takes a contiguous run of its slices (register-slice
    // and stream plans), the runs cut where the running entry count is closest to an
    // equal share
    std::vector<int32_t> wsplit(std::max<size_t>(sblk.size(), 1) * (NWARP + 1), 0);
    for (size_t bi = 0; bi < sblk.size(); ++bi) {
        const Block &bk = sblk[bi];
        if (bk.pad != 0) continue;
        const int64_t ns = bk.i1 - bk.i0, e0 = sl_base[bk.i0], tot = sl_base[bk.i1] - e0;
        int32_t *w = &wsplit[bi * (NWARP + 1)];
        int64_t q = 0;
        for (int k = 1; k < NWARP; ++k) {
            const int64_t target = e0 + tot * k / NWARP;
            while (q < ns && sl_base[bk.i0 + q + 1] <= target) ++q;
            // slice q straddles the target (or ends on it): cut before or after it
            int64_t cut = q;
            if (q < ns && sl_base[bk.i0 + q + 1] - target < target - sl_base[bk.i0 + q]) cut = q + 1;
            w[k] = (int32_t)std::max<int64_t>(cut, w[k - 1]);
        }
        w[NWARP] = (int32_t)ns;
        for (int k = 1; k < NWARP; ++k) w[k] = std::min(w[k], w[NWARP]);
    }
    // stream plans: every heavy chunk is a slice of its own after the light slices
    // (item.pad = its slice), and each warp's stream is one contiguous run of steps:
    // {first entry, steps} per (block, warp) -- its slices of a light block, or the
    // chunk it takes in a heavy block
    const int64_t n_light_slices = (int64_t)sl_base.size() - 1;
    std::vector<longlong2> wrun;
    if (tma) {
        for (SpItem &si : items) {
            si.pad = (int32_t)(sl_base.size() - 1);
            sl_base.push_back(sl_base.back() + ((si.e1 - si.e0 + H - 1) / H) * H);
            for (int r = 0; r < H; ++r) sl_row.push_back(-1);
        }
        wrun.assign(std::max<size_t>(sblk.size(), 1) * NWARP, make_longlong2(0, 0));
        for (size_t bi = 0; bi < sblk.size(); ++bi) {
            const Block &bk = sblk[bi];
            for (int k = 0; k < NWARP; ++k) {
                int64_t a = 0, z = 0;
                if (bk.pad == 0) {
                    a = sl_base[bk.i0 + wsplit[bi * (NWARP + 1) + k]];
                    z = sl_base[bk.i0 + wsplit[bi * (NWARP + 1) + k + 1]];
                } else if (bk.i0 + k < bk.i1) {
                    const int64_t sc = items[bk.i0 + k].pad;
                    a = sl_base[sc];
                    z = sl_base[sc + 1];
                }
                wrun[bi * NWARP + k] = make_longlong2(a, (z - a) / H);
            }
        }
    }
    pl->stream = tma;
    pl->tma = gm == 2;
    pl->acopy = gm == 3;
    pl->n_light_slices = n_light_slices;
    pl->n_items = (int64_t)items.size();
    pl->n_sblk = (int64_t)sblk.size();
    pl->n_heavy = nheavy;
    pl->n_chunks = nchunks;
    pl->n_vblk = (int64_t)vblk.size();
    pl->n_slices = (int64_t)sl_base.size() - 1;
    pl->n_sl_entries = sl_base.back();
    auto up = [&](DevBuf &d, const void *h, size_t bytes) -> int {
        NVD_TRY(d.alloc(bytes));
        if (bytes) NVD_TRY_CUDA(cudaMemcpy(d.p, h, bytes, cudaMemcpyHostToDevice));
        return NVD_OK;
    };
    NVD_TRY(up(pl->items, items.data(), items.size() * sizeof(SpItem)));
    NVD_TRY(up(pl->sblk, sblk.data(), sblk.size() * sizeof(Block)));
    NVD_TRY(up(pl->vblk, vblk.data(), vblk.size() * sizeof(Block)));
    NVD_TRY(up(pl->seg_sblk_off, seg_sblk_off.data(), seg_sblk_off.size() * 4));
    NVD_TRY(up(pl->seg_heavy_off, seg_heavy_off.data(), seg_heavy_off.size() * 4));
    NVD_TRY(up(pl->seg_vblk_off, seg_vblk_off.data(), seg_vblk_off.size() * 4));
    NVD_TRY(pl->hcount.alloc((size_t)std::max<int32_t>(nheavy, 1) * 4));
    NVD_TRY_CUDA(cudaMemset(pl->hcount.p, 0, pl->hcount.bytes));
    NVD_TRY(up(pl->sl_base, sl_base.data(), sl_base.size() * 8));
    NVD_TRY(up(pl->sl_wsplit, wsplit.data(), wsplit.size() * 4));
    NVD_TRY(up(pl->sl_wrun, wrun.data(), wrun.size() * sizeof(longlong2)));
    NVD_TRY(up(pl->sl_row, sl_row.data(), sl_row.size() * 4));
    // sliced weights: the graph's type (FP64 only for FP64 vectors), the solve's
    // accumulator type in stream plans (a slice's first step carries the degrees)
    const bool w64 = tma ? szv == 8 : (szv == 8 && g->wdtype == NVD_F64);
    const int64_t ne = std::max<int64_t>(pl->n_sl_entries, 1);
    NVD_TRY(pl->sl_col.alloc((size_t)ne * 4));
    NVD_TRY(pl->sl_w.alloc((size_t)ne * (w64 ? 8 : 4)));
    NVD_TRY(fill_plan_slices(g, pl.get(), 0));
    NVD_TRY_CUDA(cudaDeviceSynchronize());
    *out = pl.get();
    g->plans[key] = std::move(pl);
    return NVD_OK;
}

int get_w32(nvd_graph_s *g, const float **out, cudaStream_t s) {
    if (g->wdtype == NVD_F32) {
        *out = g->w.as<float>();
        return NVD_OK;
    }
    if (!g->w32.p) {
        const int64_t npad = ((g->nnz + 3) / 4) * 4 + 4;
        NVD_TRY(g->w32.alloc(npad * 4));
        NVD_TRY_CUDA(cudaMemsetAsync(g->w32.p, 0, npad * 4, s));
        k_round_w32<<<grid_for(g->nnz, 1, g->num_sms), 256, 0, s>>>(g->w.as<double>(),
                                                                    g->w32.as<float>(), g->nnz);
        NVD_TRY_CUDA(cudaGetLastError());
    }
    *out = g->w32.as<float>();
    return NVD_OK;
}

void set_sp_plan(Ctx *c, const Plan *pl) {
    c->items = pl->items.as<SpItem>();
    c->sblk = pl->sblk.as<Block>();
    c->n_sblk = pl->n_sblk;
    c->seg_sblk_off = pl->seg_sblk_off.as<int32_t>();
    c->seg_heavy_off = pl->seg_heavy_off.as<int32_t>();
    c->hcount = pl->hcount.as<int32_t>();
    c->sl_base = pl->sl_base.as<int64_t>();
    c->sl_row = pl->sl_row.as<int32_t>();
    c->sl_col = pl->sl_col.as<int32_t>();
    c->sl_w = pl->sl_w.p;
    c->sl_h = sp_slice_rows(pl->KT, pl->szv);
    c->sl_stream = pl->stream ? 1 : 0;
    c->sl_tma = pl->tma ? 1 : pl->acopy ? 2 : 0;
    c->sl_wsplit = pl->sl_wsplit.as<int32_t>();
    c->sl_wrun = pl->sl_wrun.as<longlong2>();
}

void fill_graph_ctx(const nvd_graph_s *g, const Plan *pl, Ctx *c) {
    c->n = g->n;
    c->rowptr = g->rowptr.as<int64_t>();
    c->colidx = g->colidx.as<int32_t>();
    c->w = g->w.p;
    c->deg64 = g->deg64.as<double>();
    c->dinv64 = g->dinv64.as<double>();
    c->deg32 = g->deg32.as<float>();
    c->dinv32 = g->dinv32.as<float>();
    c->nseg = g->nseg;
    c->seg_begin = g->seg_begin.as<int64_t>();
    c->seg_end = g->seg_end.as<int64_t>();
    c->seg_owner = g->seg_owner.as<int32_t>();
    c->perm = g->perm.as<int32_t>();
    c->hot_begin = g->hot_begin;
    c->hot_rows = g->hot_rows;
    c->l2_hot = g->sp.l2_hot;
    if (pl) {
        set_sp_plan(c, pl);
        c->vblk = pl->vblk.as<Block>();
        c->n_vblk = pl->n_vblk;
        c->seg_vblk_off = pl->seg_vblk_off.as<int32_t>();
    }
}

}  // namespace nvd

nvd_graph_s::~nvd_graph_s() {
    for (int k = 0; k < 2; ++k) {
        if (ev_copied[k]) cudaEventDestroy(ev_copied[k]);
        if (ev_used[k]) cudaEventDestroy(ev_used[k]);
    }
    if (copy_stream) cudaStreamDestroy(copy_stream);
}

void *nvd_graph_s::wsp(const std::string &name, size_t bytes, int *st) {
    auto &slot = ws[name];
    if (!slot) slot.reset(new nvd::DevBuf());
    int r = slot->ensure(bytes);
    if (r != NVD_OK) {
        *st = r;
        return nullptr;
    }
    return slot->p;
}

int64_t nvd_graph_s::device_bytes() const {
    int64_t b = 0;
    for (const nvd::DevBuf *d : {&rowptr, &colidx, &w, &w32, &deg64, &dinv64, &deg32, &dinv32,
                                 &perm, &uent, &seg_begin, &seg_end, &seg_owner})
        b += (int64_t)d->bytes;
    for (auto &kv : plans)
        for (const nvd::DevBuf *d : {&kv.second->items, &kv.second->sblk, &kv.second->vblk,
                                     &kv.second->seg_sblk_off, &kv.second->seg_heavy_off,
                                     &kv.second->seg_vblk_off, &kv.second->hcount, &kv.second->sl_base,
                                     &kv.second->sl_row, &kv.second->sl_col, &kv.second->sl_w,
                                     &kv.second->sl_wsplit, &kv.second->sl_wrun})
            b += (int64_t)d->bytes;
    for (auto &kv : ws) b += (int64_t)kv.second->bytes;
    return b;
}

// ------------------------------------------------------------------ C ABI

using namespace nvd;

static int graph_create_impl(nvd_graph_t *out, int64_t n, int64_t nnz, const int64_t *rowptr,
                             const int32_t *colidx, const void *w, int32_t wdtype, uint32_t flags,
                             cudaStream_t s) {
    if (n < 1 || n > INT32_MAX - 1 || nnz < 0 || !rowptr || (nnz > 0 && !colidx) ||
        (wdtype != NVD_F32 && wdtype != NVD_F64) ||
        (flags & ~(NVD_GRAPH_DEVICE_PTRS | NVD_GRAPH_SKIP_SYM_CHECK | NVD_GRAPH_REORDER_DEGREE))) {
        set_error("nvd_graph_create: invalid argument (n=%lld nnz=%lld wdtype=%d flags=%u)",
                  (long long)n, (long long)nnz, wdtype, flags);
        return NVD_ERR_INVALID_ARG;
    }
    const bool dev = flags & NVD_GRAPH_DEVICE_PTRS;
    std::unique_ptr<nvd_graph_s> g(new nvd_graph_s());
    g->id = next_graph_id();
    NVD_TRY_CUDA(cudaGetDevice(&g->device));
    NVD_TRY_CUDA(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device));
    g->n = n;
    g->nnz = nnz;
    g->nnz_user = nnz;
    g->wdtype = wdtype;
    const size_t wsz = wdtype == NVD_F64 ? 8 : 4;

    // rowptr: host copy (planning) and validation
    g->h_rowptr.resize(n + 1);
    if (dev)
        NVD_TRY_CUDA(cudaMemcpyAsync(g->h_rowptr.data(), rowptr, (n + 1) * 8, cudaMemcpyDeviceToHost, s));
    else
        memcpy(g->h_rowptr.data(), rowptr, (n + 1) * 8);
    NVD_TRY_CUDA(cudaStreamSynchronize(s));
    if (g->h_rowptr[0] != 0 || g->h_rowptr[n] != nnz) {
        set_error("nvd_graph_create: rowptr[0] must be 0 and rowptr[n] must equal nnz");
        return NVD_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < n; ++i)
        if (g->h_rowptr[i + 1] < g->h_rowptr[i]) {
            set_error("nvd_graph_create: rowptr decreases at row %lld", (long long)i);
            return NVD_ERR_INVALID_ARG;
        }

    // device copies (padded to a multiple of 4 entries for 16-byte loads)
    const int64_t npad = ((nnz + 3) / 4) * 4 + 4;
    NVD_TRY(g->rowptr.alloc((n + 1) * 8));
    NVD_TRY_CUDA(cudaMemcpyAsync(g->rowptr.p, g->h_rowptr.data(), (n + 1) * 8, cudaMemcpyHostToDevice, s));
    NVD_TRY(g->colidx.alloc(npad * 4));
    NVD_TRY_CUDA(cudaMemsetAsync(g->colidx.p, 0, npad * 4, s));
    NVD_TRY(g->w.alloc(npad * wsz));
    NVD_TRY_CUDA(cudaMemsetAsync(g->w.p, 0, npad * wsz, s));
    if (nnz > 0) {
        const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        NVD_TRY_CUDA(cudaMemcpyAsync(g->colidx.p, colidx, nnz * 4, kind, s));
        if (w) {
            NVD_TRY_CUDA(cudaMemcpyAsync(g->w.p, w, nnz * wsz, kind, s));
        } else if (wdtype == NVD_F64) {
            k_fill<double><<<grid_for(nnz, 1, g->num_sms), 256, 0, s>>>(g->w.as<double>(), nnz, 1.0);
        } else {
            k_fill<float><<<grid_for(nnz, 1, g->num_sms), 256, 0, s>>>(g->w.as<float>(), nnz, 1.0f);
        }
        NVD_TRY_CUDA(cudaGetLastError());
    }

    // structure and weight checks
    int fl[4] = {0, 0, 0, 0};
    if (wdtype == NVD_F64)
        NVD_TRY(run_checks<double>(g.get(), w != nullptr, fl, s));
    else
        NVD_TRY(run_checks<float>(g.get(), w != nullptr, fl, s));
    if (fl[0]) {
        set_error("nvd_graph_create: column index out of range");
        return NVD_ERR_INVALID_ARG;
    }
    if (fl[3]) {
        set_error("nvd_graph_create: weights must be finite and > 0");
        return NVD_ERR_BAD_WEIGHT;
    }
    std::vector<int64_t> uent;  // user entry -> internal entry, empty = identity
    if (fl[1] || fl[2]) {
        std::vector<int32_t> col;
        std::vector<double> wv;
        NVD_TRY(download_csr(g.get(), col, wv, s));
        HostCSR hc;
        clean_csr(n, g->h_rowptr, col, wv, hc);
        g->nnz = (int64_t)hc.col.size();
        g->h_rowptr = hc.rowptr;
        uent = hc.uent;
        NVD_TRY_CUDA(cudaMemcpyAsync(g->rowptr.p, g->h_rowptr.data(), (n + 1) * 8, cudaMemcpyHostToDevice, s));
        NVD_TRY(upload_padded(g->colidx, hc.col.data(), g->nnz, s));
        NVD_TRY(upload_weights(g.get(), hc.w, s));
        NVD_TRY_CUDA(cudaStreamSynchronize(s));
    }
    if (!(flags & NVD_GRAPH_SKIP_SYM_CHECK)) {
        int bad = 0;
        if (wdtype == NVD_F64)
            NVD_TRY(run_sym<double>(g.get(), &bad, s));
        else
            NVD_TRY(run_sym<float>(g.get(), &bad, s));
        if (bad) {
            set_error("nvd_graph_create: the CSR is not symmetric (structure or weights)");
            return NVD_ERR_NOT_SYMMETRIC;
        }
    }

    // connected components; relabel if some component is not a contiguous range
    std::vector<int32_t> root;
    NVD_TRY(run_components(g.get(), root, s));
    std::vector<int64_t> cnt(n, 0), mx(n, -1);
    for (int64_t i = 0; i < n; ++i) {
        cnt[root[i]]++;
        mx[root[i]] = std::max<int64_t>(mx[root[i]], i);
    }
    bool contiguous = true;
    int32_t ncomp = 0;
    for (int64_t r = 0; r < n; ++r)
        if (cnt[r] > 0) {
            ++ncomp;
            if (mx[r] - r + 1 != cnt[r]) contiguous = false;
        }
    g->ncomp = ncomp;
    std::vector<int32_t> perm;  // internal -> user
    const bool reorder = flags & NVD_GRAPH_REORDER_DEGREE;
    if (!contiguous || reorder) {
        // stable counting sort of nodes by their component's smallest node; with
        // NVD_GRAPH_REORDER_DEGREE each component's nodes then by stored entries,
        // most first (ties by node), so its most gathered rows are one contiguous run
        std::vector<int64_t> start(n + 1, 0);
        for (int64_t r = 0; r < n; ++r) start[r + 1] = start[r] + cnt[r];
        perm.resize(n);
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int64_t i = 0; i < n; ++i) perm[fill[root[i]]++] = (int32_t)i;
        if (reorder) {
            const std::vector<int64_t> &rp = g->h_rowptr;
            for (int64_t r = 0; r < n; ++r)
                if (cnt[r] > 1)
                    std::stable_sort(perm.begin() + start[r], perm.begin() + start[r + 1], [&](int32_t a, int32_t b) {
                        return rp[a + 1] - rp[a] > rp[b + 1] - rp[b];
                    });
        }
        std::vector<int32_t> iperm(n);
        for (int64_t i = 0; i < n; ++i) iperm[perm[i]] = (int32_t)i;
        std::vector<int32_t> col;
        std::vector<double> wv;
        NVD_TRY(download_csr(g.get(), col, wv, s));
        std::vector<int64_t> rp2(n + 1, 0);
        for (int64_t i = 0; i < n; ++i)
            rp2[i + 1] = rp2[i] + (g->h_rowptr[perm[i] + 1] - g->h_rowptr[perm[i]]);
        std::vector<int32_t> col2(g->nnz);
        std::vector<double> w2(g->nnz);
        std::vector<int64_t> newpos(g->nnz);
        std::vector<std::pair<int32_t, int64_t>> tmp;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t u = perm[i];
            tmp.clear();
            for (int64_t e = g->h_rowptr[u]; e < g->h_rowptr[u + 1]; ++e) tmp.push_back({iperm[col[e]], e});
            std::sort(tmp.begin(), tmp.end());
            for (size_t t = 0; t < tmp.size(); ++t) {
                const int64_t pos = rp2[i] + (int64_t)t;
                col2[pos] = tmp[t].first;
                w2[pos] = wv[tmp[t].second];
                newpos[tmp[t].second] = pos;
            }
        }
        if (uent.empty()) {
            uent.resize(g->nnz_user);
            for (int64_t e = 0; e < g->nnz_user; ++e) uent[e] = newpos[e];
        } else {
            for (int64_t e = 0; e < g->nnz_user; ++e)
                if (uent[e] >= 0) uent[e] = newpos[uent[e]];
        }
        g->h_rowptr = rp2;
        NVD_TRY_CUDA(cudaMemcpyAsync(g->rowptr.p, g->h_rowptr.data(), (n + 1) * 8, cudaMemcpyHostToDevice, s));
        NVD_TRY(upload_padded(g->colidx, col2.data(), g->nnz, s));
        NVD_TRY(upload_weights(g.get(), w2, s));
        NVD_TRY(g->perm.alloc(n * 4));
        NVD_TRY_CUDA(cudaMemcpyAsync(g->perm.p, perm.data(), n * 4, cudaMemcpyHostToDevice, s));
        // roots in the new order
        std::vector<int32_t> root2(n);
        for (int64_t i = 0; i < n; ++i) root2[i] = iperm[root[perm[i]]];
        // in the new order every component is one run of equal labels
        root.swap(root2);
        NVD_TRY_CUDA(cudaStreamSynchronize(s));
    }
    if (!uent.empty()) {
        NVD_TRY(g->uent.alloc(uent.size() * 8));
        NVD_TRY_CUDA(cudaMemcpyAsync(g->uent.p, uent.data(), uent.size() * 8, cudaMemcpyHostToDevice, s));
    }
    // segments: contiguous runs of equal component with >= 2 nodes
    {
        int64_t i = 0;
        while (i < n) {
            int64_t j = i + 1;
            while (j < n && root[j] == root[i]) ++j;
            if (j - i >= 2) {
                g->h_seg_begin.push_back(i);
                g->h_seg_end.push_back(j);
            } else {
                g->n_singleton++;
            }
            i = j;
        }
    }
    g->nseg = (int32_t)g->h_seg_begin.size();
    if (reorder && g->nseg > 0) {
        g->reordered = true;
        int32_t big = 0;
        for (int32_t sg = 1; sg < g->nseg; ++sg)
            if (g->h_seg_end[sg] - g->h_seg_begin[sg] > g->h_seg_end[big] - g->h_seg_begin[big]) big = sg;
        g->hot_begin = g->h_seg_begin[big];
        g->hot_rows = g->h_seg_end[big] - g->h_seg_begin[big];
    }
    g->h_seg_of.assign(n, -1);
    for (int32_t sg = 0; sg < g->nseg; ++sg)
        for (int64_t i = g->h_seg_begin[sg]; i < g->h_seg_end[sg]; ++i)
            g->h_seg_of[perm.empty() ? i : perm[i]] = sg;
    const size_t ns = std::max<size_t>(g->h_seg_begin.size(), 1);
    NVD_TRY(g->seg_begin.alloc(ns * 8));
    NVD_TRY(g->seg_end.alloc(ns * 8));
    NVD_TRY(g->seg_owner.alloc(ns * 4));
    NVD_TRY_CUDA(cudaMemsetAsync(g->seg_owner.p, 0, ns * 4, s));
    if (g->nseg) {
        NVD_TRY_CUDA(cudaMemcpyAsync(g->seg_begin.p, g->h_seg_begin.data(), g->nseg * 8, cudaMemcpyHostToDevice, s));
        NVD_TRY_CUDA(cudaMemcpyAsync(g->seg_end.p, g->h_seg_end.data(), g->nseg * 8, cudaMemcpyHostToDevice, s));
    }
    NVD_TRY(run_degree(g.get(), s));
    NVD_TRY_CUDA(cudaStreamSynchronize(s));
    *out = g.release();
    return NVD_OK;
}

extern "C" int nvd_graph_create(nvd_graph_t *out, int64_t n, int64_t nnz, const int64_t *rowptr,
                                const int32_t *colidx, const void *w, int32_t wdtype, uint32_t flags,
                                nvd_stream_t stream) {
    clear_error();
    if (!out) {
        set_error("nvd_graph_create: out is NULL");
        return NVD_ERR_INVALID_ARG;
    }
    *out = nullptr;
    try {
        return graph_create_impl(out, n, nnz, rowptr, colidx, w, wdtype, flags, (cudaStream_t)stream);
    } catch (const std::bad_alloc &) {
        set_error("nvd_graph_create: host allocation failed");
        return NVD_ERR_OOM;
    } catch (...) {
        set_error("nvd_graph_create: unexpected host exception");
        return NVD_ERR_CUDA;
    }
}

// New weights for the same sparsity pattern: validate them, map them onto the
// handle's entries (repeated entries summed, self-loops dropped, node relabelling
// applied, as at creation), check symmetry, then replace the weights, the degrees,
// the FP32 copy and the sliced copies of every cached plan.  Nothing is replaced
// when a check fails.
static int set_weights_impl(nvd_graph_t g, const void *w, int32_t wdtype, uint32_t flags, cudaStream_t s) {
    if (!g || !w || wdtype != g->wdtype || (flags & ~(NVD_GRAPH_DEVICE_PTRS | NVD_GRAPH_SKIP_SYM_CHECK))) {
        set_error("nvd_graph_set_weights: invalid argument (the weight type must be the handle's, %s)",
                  g && g->wdtype == NVD_F64 ? "NVD_F64" : "NVD_F32");
        return NVD_ERR_INVALID_ARG;
    }
    const size_t wsz = g->wdtype == NVD_F64 ? 8 : 4;
    const int64_t nu = g->nnz_user, ni = g->nnz;
    int st = NVD_OK;
    void *wu = g->wsp("setw_user", (size_t)std::max<int64_t>(nu, 1) * wsz, &st);
    const int64_t npad = ((ni + 3) / 4) * 4 + 4;
    void *wi = g->wsp("setw_new", (size_t)npad * wsz, &st);
    int *flag = (int *)g->wsp("setw_flag", 16, &st);
    if (st) return st;
    if (nu > 0)
        NVD_TRY_CUDA(cudaMemcpyAsync(wu, w, (size_t)nu * wsz,
                                     (flags & NVD_GRAPH_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    NVD_TRY_CUDA(cudaMemsetAsync(flag, 0, 16, s));
    NVD_TRY_CUDA(cudaMemsetAsync(wi, 0, (size_t)npad * wsz, s));
    const int grid = grid_for(std::max<int64_t>(nu, ni), 1, g->num_sms);
    if (nu > 0) {
        if (g->wdtype == NVD_F64)
            k_check_weights<double><<<grid, 256, 0, s>>>(nu, (const double *)wu, flag);
        else
            k_check_weights<float><<<grid, 256, 0, s>>>(nu, (const float *)wu, flag);
        NVD_TRY_CUDA(cudaGetLastError());
    }
    int bad_w = 0;
    NVD_TRY_CUDA(cudaMemcpyAsync(&bad_w, flag, 4, cudaMemcpyDeviceToHost, s));
    NVD_TRY_CUDA(cudaStreamSynchronize(s));
    if (bad_w) {
        set_error("nvd_graph_set_weights: weights must be finite and > 0");
        return NVD_ERR_BAD_WEIGHT;
    }
    if (ni > 0) {
        if (!g->uent.p) {
            NVD_TRY_CUDA(cudaMemcpyAsync(wi, wu, (size_t)ni * wsz, cudaMemcpyDeviceToDevice, s));
        } else {
            if (!g->ient_ptr.p) {
                std::vector<int64_t> ue(nu);
                NVD_TRY_CUDA(cudaMemcpyAsync(ue.data(), g->uent.p, (size_t)nu * 8, cudaMemcpyDeviceToHost, s));
                NVD_TRY_CUDA(cudaStreamSynchronize(s));
                std::vector<int64_t> ptr(ni + 1, 0), src;
                for (int64_t e = 0; e < nu; ++e)
                    if (ue[e] >= 0) ++ptr[ue[e] + 1];
                for (int64_t e = 0; e < ni; ++e) ptr[e + 1] += ptr[e];
                src.resize(std::max<int64_t>(ptr[ni], 1));
                std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
                for (int64_t e = 0; e < nu; ++e)
                    if (ue[e] >= 0) src[fill[ue[e]]++] = e;
                NVD_TRY(g->ient_ptr.alloc((size_t)(ni + 1) * 8));
                NVD_TRY(g->ient_src.alloc(src.size() * 8));
                NVD_TRY_CUDA(cudaMemcpyAsync(g->ient_ptr.p, ptr.data(), (size_t)(ni + 1) * 8, cudaMemcpyHostToDevice, s));
                NVD_TRY_CUDA(cudaMemcpyAsync(g->ient_src.p, src.data(), src.size() * 8, cudaMemcpyHostToDevice, s));
                NVD_TRY_CUDA(cudaStreamSynchronize(s));
            }
            if (g->wdtype == NVD_F64)
                k_gather_weights<double><<<grid, 256, 0, s>>>(ni, g->ient_ptr.as<int64_t>(), g->ient_src.as<int64_t>(),
                                                              (const double *)wu, (double *)wi);
            else
                k_gather_weights<float><<<grid, 256, 0, s>>>(ni, g->ient_ptr.as<int64_t>(), g->ient_src.as<int64_t>(),
                                                             (const float *)wu, (float *)wi);
            NVD_TRY_CUDA(cudaGetLastError());
        }
        if (!(flags & NVD_GRAPH_SKIP_SYM_CHECK)) {
            int bad = 0;
            if (g->wdtype == NVD_F64)
                NVD_TRY(run_sym<double>(g, &bad, s, (const double *)wi));
            else
                NVD_TRY(run_sym<float>(g, &bad, s, (const float *)wi));
            if (bad) {
                set_error("nvd_graph_set_weights: the new weights are not symmetric");
                return NVD_ERR_NOT_SYMMETRIC;
            }
        }
    }
    // commit
    NVD_TRY_CUDA(cudaMemcpyAsync(g->w.p, wi, (size_t)npad * wsz, cudaMemcpyDeviceToDevice, s));
    NVD_TRY(run_degree(g, s));
    if (g->w32.p && g->wdtype == NVD_F64 && ni > 0) {
        k_round_w32<<<grid_for(ni, 1, g->num_sms), 256, 0, s>>>(g->w.as<double>(), g->w32.as<float>(), ni);
        NVD_TRY_CUDA(cudaGetLastError());
    }
    for (auto &kv : g->plans) NVD_TRY(fill_plan_slices(g, kv.second.get(), s));
    NVD_TRY_CUDA(cudaStreamSynchronize(s));
    g->elim.reset();            // the reduced graph depends on the weights
    g->id = next_graph_id();    // caches keyed by the handle (batched unions, captured launches) miss
    return NVD_OK;
}

extern "C" int nvd_graph_set_weights(nvd_graph_t g, const void *w, int32_t wdtype, uint32_t flags,
                                     nvd_stream_t stream) {
    clear_error();
    if (!g) {
        set_error("nvd_graph_set_weights: NULL handle");
        return NVD_ERR_INVALID_ARG;
    }
    try {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != g->device) cudaSetDevice(g->device);
        const int rc = set_weights_impl(g, w, wdtype, flags, (cudaStream_t)stream);
        if (cur >= 0 && cur != g->device) cudaSetDevice(cur);
        return rc;
    } catch (const std::bad_alloc &) {
        set_error("nvd_graph_set_weights: host allocation failed");
        return NVD_ERR_OOM;
    } catch (...) {
        set_error("nvd_graph_set_weights: unexpected host exception");
        return NVD_ERR_CUDA;
    }
}

extern "C" int nvd_graph_destroy(nvd_graph_t g) {
    clear_error();
    if (!g) return NVD_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(g->device);
    delete g;
    cudaSetDevice(dev);
    return NVD_OK;
}

extern "C" int nvd_graph_info(nvd_graph_t g, int64_t *n, int64_t *nnz, int32_t *ncomp,
                              int64_t *device_bytes) {
    clear_error();
    if (!g) {
        set_error("nvd_graph_info: NULL handle");
        return NVD_ERR_INVALID_ARG;
    }
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (ncomp) *ncomp = g->ncomp;
    if (device_bytes) *device_bytes = g->device_bytes();
    return NVD_OK;
}
