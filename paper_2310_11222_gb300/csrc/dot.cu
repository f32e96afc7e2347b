// C ABI: nvd_dot_f32 -- the FP32-mode inner product of the solver on its own.
//
// FP32-mode PCG keeps its vectors in FP32 but takes every inner product (p^T q,
// r^T D^-1 r, |r|^2) with a per-thread double-float accumulator fed with the
// exact product of two floats, then FP64 block and cross-block sums in a fixed
// order.  This entry point runs exactly that reduction on two FP32 vectors, so
// its accuracy can be checked against an exact sum (and used by callers who need
// an accurate FP32 dot product).
#include <algorithm>

#include "graph.h"
#include "kernels.cuh"

namespace nvd {
void note_launch(int64_t n);
}

namespace {

using namespace nvd;

constexpr int DOT_BLOCKS_MAX = 1024;

__global__ void __launch_bounds__(NT) k_dot_f32_part(const float *__restrict__ a, const float *__restrict__ b,
                                                     int64_t n, double *__restrict__ part) {
    __shared__ double red[red_doubles(1)];
    __shared__ double tot[4];
    dev::DFloat acc;
    dev::dot_zero(acc);
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT)
        dev::dot_fma(acc, __ldg(a + i), __ldg(b + i));
    double dd[1][1] = {{dev::dot_get(acc)}};
    dev::block_reduce_cols<1, 1, 1>(dd, red, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot[0];
}

// The block totals in block order.
__global__ void k_dot_f32_final(const double *__restrict__ part, int nb, double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += part[i];
        *out = s;
    }
}

int dot_impl(const float *a, const float *b, int64_t n, double *out, cudaStream_t s) {
    if (n < 0 || !out || (n > 0 && (!a || !b))) {
        set_error("nvd_dot_f32: invalid argument");
        return NVD_ERR_INVALID_ARG;
    }
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n + NT - 1) / NT, DOT_BLOCKS_MAX));
    double *part = nullptr;
    NVD_TRY_CUDA(cudaMallocAsync((void **)&part, (size_t)nb * sizeof(double), s));
    if (n > 0) {
        k_dot_f32_part<<<nb, NT, 0, s>>>(a, b, n, part);
    } else {
        cudaMemsetAsync(part, 0, sizeof(double), s);
    }
    k_dot_f32_final<<<1, 32, 0, s>>>(part, nb, out);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(part, s);
    if (e != cudaSuccess) {
        set_error("nvd_dot_f32: %s", cudaGetErrorString(e));
        return NVD_ERR_CUDA;
    }
    note_launch(n > 0 ? 2 : 1);
    return NVD_OK;
}

}  // namespace

extern "C" int nvd_dot_f32(const float *a, const float *b, int64_t n, double *out, nvd_stream_t stream) {
    clear_error();
    try {
        return dot_impl(a, b, n, out, (cudaStream_t)stream);
    } catch (...) {
        set_error("nvd_dot_f32: unexpected host exception");
        return NVD_ERR_CUDA;
    }
}
