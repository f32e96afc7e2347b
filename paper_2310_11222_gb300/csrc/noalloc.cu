// C ABI: nvd_laplacian_quadform_noalloc -- y = L x and x^T L x with no allocation.
//
// A variant of the Laplacian SpMV with its fused inner product (the kernel the
// PCG runs every iteration) for callers that cannot allocate device memory at
// call time: for example a process whose device memory is already reserved by
// another framework's caching allocator, or a latency-critical loop where an
// allocation (and the device-wide synchronisation it can imply) is not allowed.
// The graph handle is created beforehand (nvd_graph_create allocates); this call
// itself allocates nothing: its cross-block partial sums live in the file-scope
// device array below, which every GPU that loads the library holds until the
// process exits.
#include <mutex>

#include "graph.h"

namespace {

constexpr int NA_MAX_K = 32;        // columns per call
constexpr int NA_MAX_BLOCKS = 1024; // CTAs per call (partial-sum slots)
constexpr int NA_THREADS = 256;
// [NA_MAX_BLOCKS][NA_MAX_K] doubles of block partial sums, then one arrival counter.
constexpr size_t NA_PART_BYTES = (size_t)NA_MAX_BLOCKS * NA_MAX_K * sizeof(double);
constexpr size_t NA_SCRATCH_BYTES = NA_PART_BYTES + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device (host code must not use the
// symbol itself: on the host it only names a stand-in, not device memory).
std::mutex g_na_mu;
void *g_na_addr[128] = {nullptr};

int scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= 128) {
        nvd::set_error("nvd_laplacian_quadform_noalloc: device ordinal %d out of range", dev);
        return NVD_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            nvd::set_error("nvd_laplacian_quadform_noalloc: cudaGetSymbolAddress failed: %s",
                           cudaGetErrorString(e));
            return NVD_ERR_CUDA;
        }
        g_na_addr[dev] = p;
    }
    *out = g_na_addr[dev];
    return NVD_OK;
}

// One warp per row (grid-stride), lanes striding over the row's entries; x, y in
// the caller's node order ([k][n]), the CSR in the handle's internal order.
template <class TW>
__global__ void __launch_bounds__(NA_THREADS)
k_quadform_noalloc(int64_t n, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                   const TW *__restrict__ w, const double *__restrict__ deg, const int32_t *__restrict__ perm,
                   int k, const double *__restrict__ x, double *__restrict__ y, double *__restrict__ q,
                   unsigned char *scratch) {
    double *part = reinterpret_cast<double *>(scratch);
    unsigned *count = reinterpret_cast<unsigned *>(scratch + NA_PART_BYTES);
    __shared__ double red[NA_THREADS / 32];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int j = 0; j < k; ++j) {
        const double *xj = x + (int64_t)j * n;
        double dot = 0.0;
        for (int64_t i = warp; i < n; i += nw) {
            const int64_t u = perm ? (int64_t)perm[i] : i;
            double s = 0.0;
            for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
                const int32_t v = colidx[e];
                s += (double)w[e] * xj[perm ? (int64_t)perm[v] : (int64_t)v];
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) {
                const double xu = xj[u];
                const double val = deg[i] * xu - s;
                if (y) y[(int64_t)j * n + u] = val;
                dot += xu * val;
            }
        }
        if (lane == 0) red[wib] = dot;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q2 = 0; q2 < NA_THREADS / 32; ++q2) t += red[q2];
            part[(int64_t)blockIdx.x * NA_MAX_K + j] = t;
        }
        __syncthreads();
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(count, 1u) == gridDim.x - 1);
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (threadIdx.x < k) {
            double t = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(part + (int64_t)b * NA_MAX_K + threadIdx.x);
            q[threadIdx.x] = t;
        }
        if (threadIdx.x == 0) atomicExch(count, 0u);
    }
}

}  // namespace

extern "C" int nvd_laplacian_quadform_noalloc(nvd_graph_t g, int32_t k, const double *x, double *y,
                                              double *q, nvd_stream_t stream) {
    nvd::clear_error();
    if (!g || k < 1 || !x || !q) {
        nvd::set_error("nvd_laplacian_quadform_noalloc: invalid argument");
        return NVD_ERR_INVALID_ARG;
    }
    if (k > NA_MAX_K) {
        nvd::set_error("nvd_laplacian_quadform_noalloc: k = %d exceeds the maximum of %d columns per call", k,
                       NA_MAX_K);
        return NVD_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != g->device) cudaSetDevice(g->device);
    int rc = NVD_OK;
    void *scratch = nullptr;
    rc = scratch_address(g->device, &scratch);
    if (rc == NVD_OK) {
        int64_t blocks = ((int64_t)g->n * 32 + NA_THREADS - 1) / NA_THREADS;
        if (blocks > NA_MAX_BLOCKS) blocks = NA_MAX_BLOCKS;
        if (blocks > (int64_t)g->num_sms * 8) blocks = (int64_t)g->num_sms * 8;
        if (blocks < 1) blocks = 1;
        // the arrival counter must start at zero (a previous call on this device
        // leaves it at zero, an interrupted one may not)
        cudaError_t e = cudaMemsetAsync((unsigned char *)scratch + NA_PART_BYTES, 0, sizeof(unsigned), s);
        if (e == cudaSuccess) {
            if (g->wdtype == NVD_F64)
                k_quadform_noalloc<double><<<(unsigned)blocks, NA_THREADS, 0, s>>>(
                    g->n, g->rowptr.as<int64_t>(), g->colidx.as<int32_t>(), g->w.as<double>(), g->deg64.as<double>(),
                    g->perm.as<int32_t>(), k, x, y, q, (unsigned char *)scratch);
            else
                k_quadform_noalloc<float><<<(unsigned)blocks, NA_THREADS, 0, s>>>(
                    g->n, g->rowptr.as<int64_t>(), g->colidx.as<int32_t>(), g->w.as<float>(), g->deg64.as<double>(),
                    g->perm.as<int32_t>(), k, x, y, q, (unsigned char *)scratch);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            nvd::set_error("nvd_laplacian_quadform_noalloc: %s", cudaGetErrorString(e));
            rc = NVD_ERR_CUDA;
        }
    }
    if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
    return rc;
}
